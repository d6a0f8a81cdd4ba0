/*
 * cb_uniform.h -- uniform single trades of libcb.so: the Simple Undirected
 * Curveball chain (Section 3.2), whose trades are node pairs drawn uniformly
 * at random and applied one after the other, and the successor lists Suc of
 * a trade sequence (Section 4.1).
 *
 * Trade i (0-based, 64-bit index) of the sequence of a seed:
 *   - its pair: Philox4x32-10 (the generator of cb.h) on counter
 *     (i_lo, i_hi, 0, 5) gives r0..r3; u = floor(r0 n / 2^32),
 *     w = floor(r1 (n-1) / 2^32), v = w + (w >= u).  So u != v, and every
 *     ordered pair has probability 1/(n(n-1)) up to a relative 2^-32.
 *   - its shuffle: every disjoint neighbour x (node id) of u and v gets the
 *     key (r0 << 32 | r1) of Philox4x32-10 on counter (x, i_lo, i_hi, 6);
 *     sigma(D) is D sorted by (key, x), and u receives its first |A_{u-v}|
 *     elements (Fig. 2).
 * The result after any number of trades is bit-identical to applying them
 * one after another in index order.
 *
 * On the device the sequence runs as a dataflow in the manner of EM-CB and
 * IM-CB (Sections 4.1-4.2):
 *   - every edge waits in the inbox of the next trade of either endpoint,
 *     found through Suc;
 *   - a trade runs as soon as its inboxes hold both degrees' worth of edges;
 *   - it then sends each resulting edge on to the next trade of either
 *     endpoint, or writes it out when neither endpoint trades again.
 * Conventions (sizes, return codes, streams) are those of cb.h.
 */
#ifndef CB_UNIFORM_H
#define CB_UNIFORM_H

#include <stdint.h>

#include "cb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Apply the handle's next `count` uniform trades (indices next .. next +
 * count - 1, where next is what cb_uniform_next reports; it starts at 0 for
 * a new handle).  The graph state is replaced by the result.  Global super
 * steps and uniform trades may alternate freely: each kind keeps its own
 * index.
 *
 * Work and memory:
 *   - The sequence is processed in chunks of at most max(n/2, 65536) trades.
 *   - A chunk holds one 8-byte inbox slot per (trade, endpoint, neighbour),
 *     about 16 m bytes for n/2 trades.
 *   - The call synchronises the handle's stream once per chunk.
 *
 * Errors:
 *   - With n < 2 no pair exists: the index advances and the graph is
 *     unchanged.
 *   - Handles of several graphs (cb_create_batch) return CB_EINVAL.
 *   - A device wait that exceeds 20 s, or an inbox or row overflow, latches
 *     CB_ECHECK.
 */
int cb_uniform_trades(cb_handle h, uint64_t count);

/* Index of the handle's next uniform trade. */
int cb_uniform_next(cb_handle h, uint64_t* next);

/*
 * Node pairs of uniform trades first .. first + count - 1 of `seed` on n >= 2
 * nodes: pairs[2k] = u and pairs[2k+1] = v of trade first + k.  pairs is
 * device memory (2 count int32).  The call does not synchronise.
 */
int cb_uniform_pairs(uint64_t seed, int64_t n, uint64_t first, int64_t count, int32_t* pairs, void* cuda_stream);

/*
 * Successor lists (Section 4.1) of the trade sequence t_i = {pairs[2i],
 * pairs[2i+1]}, i < count:
 *   - node x's trades are suc[suc_begin[x] .. suc_begin[x+1]), in
 *     increasing order;
 *   - the closing "infinity" of the paper is the end of that range.
 * All buffers are device memory:
 *   - pairs: 2 count int32;
 *   - suc_begin: n+1 int64;
 *   - suc: 2 count int32.
 * Returns CB_EINVAL for a node outside [0, n) or a pair of equal nodes.
 * Synchronises the stream.
 */
int cb_successors(int64_t n, const int32_t* pairs, int64_t count, int64_t* suc_begin, int32_t* suc,
                  void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CB_UNIFORM_H */
