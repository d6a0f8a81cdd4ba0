/*
 * cb_gen.h -- seeded input graphs generated on the device (libcb.so).
 *
 * The inputs of the paper's experiments are power-law degree sequences
 * (Section 2, "Randomisation and Distributions": PLD([a,b), gamma),
 * P[X = k] proportional to k^-gamma for a <= k < b) realised as simple graphs
 * by Havel-Hakimi (Section 5.2).  These calls produce exactly the graphs of
 * the host generator the tests and benchmarks use (byte for byte: the same
 * draws, the same table, the same Havel-Hakimi tie order), in device memory.
 * Return codes and errors as in cb.h (cb_last_error(NULL) describes them).
 */
#ifndef CB_GEN_H
#define CB_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * n i.i.d. degrees from PLD([a,b), gamma) into deg_out (n int32, device
 * memory, caller-owned): degree i is the smallest k in [a, b) whose
 * cumulative weight exceeds u_i times the total weight, u_i the i-th
 * uniform draw (53 bits, SplitMix64 stream 0 of `seed`); if the degrees sum
 * to an odd number, the last one gets one more.  *sum_out receives the sum.
 * CB_EINVAL for n < 0, a < 0, b <= a or gamma < 1.  Runs on cuda_stream
 * (NULL: the default stream) and waits for it.
 */
int cb_generate_pld(int64_t n, int32_t a, int32_t b, double gamma, uint64_t seed, int32_t* deg_out,
                    int64_t* sum_out, void* cuda_stream);

/*
 * Havel-Hakimi realisation of the degree sequence deg (n int32, device
 * memory): repeatedly the node of largest residual degree d (the first in
 * the residual order) is joined to the next d nodes of that order, and the
 * order is updated as by the host generator (nodes first ordered by
 * descending degree, ties by id).  Writes row_ptr (n+1 int64) and col
 * (sum of degrees int32), device memory, caller-owned, rows ascending;
 * *m_out = the number of edges.  CB_EINVAL if the sequence is not graphical
 * (the greedy fails, the sum is odd, or a degree lies outside [0, n));
 * CB_ESIZE for a degree above 16384.  The greedy's steps depend on each
 * other, so one warp runs them; their connections and the CSR are built in
 * parallel.  Allocates scratch of about 12 bytes per node and 8 per edge on
 * cuda_stream (NULL: the default stream) and waits for it.
 */
int cb_generate_hh(int64_t n, const int32_t* deg, int64_t* row_ptr, int32_t* col, int64_t* m_out,
                   void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CB_GEN_H */
