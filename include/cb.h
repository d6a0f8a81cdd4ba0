/*
 * cb.h -- C ABI of the GB300 global Curveball library (libcb.so).
 *
 * The library randomises a simple undirected graph with the undirected global
 * Curveball chain of Carstens, Hamann, Meyer, Penschuck, Tran and Wagner,
 * "Parallel and I/O-efficient Randomisation of Massive Networks using Global
 * Curveball Trades":
 *   - Def. "Simple Undirected Trade" (Section 3.2, Fig. 2): nodes u and v keep
 *     their common neighbours; their disjoint neighbours D are shuffled and
 *     dealt back so that both degrees are kept;
 *   - Def. "Undirected Global Trade" (Section 3.3): a random permutation pi
 *     pairs the nodes into floor(n/2) trades applied in index order (one
 *     "super step");
 *   - Section 4: the algorithm draws each trade's shuffle itself.
 * The result of every super step is bit-identical to applying the trades one
 * after another in index order; how the permutation and shuffles are drawn
 * from (seed, super-step index) is fixed below (see cb_global_trades).
 *
 * Conventions for every entry point:
 *   - Sizes are 64-bit; node ids are int32 in [0, n); n <= 2^31 - 1; the
 *     number of undirected edges m must be < 2^32 and every node's degree
 *     < n.
 *   - mem_kind says where a caller buffer lives: CB_HOST (pageable or pinned
 *     host memory) or CB_DEVICE (device memory of the current CUDA device,
 *     e.g. a torch tensor's data_ptr()).
 *   - Return codes: CB_OK (0) or a negative CB_E* code.  Nothing aborts or
 *     traps; after an error cb_last_error() describes it.  An error latched
 *     by a device check (CB_ECHECK) or by a device wait that ran out
 *     (CB_ETIMEOUT) makes later calls on the handle fail; cb_destroy still
 *     releases it.  Every device-side wait (a trade waiting for the trade it
 *     depends on, a bulk copy into shared memory, the uniform-trade
 *     executor's run queue and inboxes) is bounded in time (option
 *     "wait_ms"); the kernel then records the error and returns.
 *   - One host thread at a time per handle.  Work is issued on the handle's
 *     stream; calls that return data to the caller synchronise that stream.
 */
#ifndef CB_H
#define CB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CB_OK 0
#define CB_EINVAL (-1)   /* bad argument or graph not simple / not symmetric */
#define CB_ENOMEM (-2)   /* device or host allocation failed */
#define CB_ECUDA (-3)    /* a CUDA runtime call failed */
#define CB_ECHECK (-5)   /* a device-side invariant check failed */
#define CB_ESIZE (-6)    /* caller buffer too small (size reported) */
#define CB_ERANGE (-7)   /* super-step counter would exceed 2^32 - 2 */
#define CB_ETIMEOUT (-8) /* a bounded device wait ran out (the handle stays destroyable) */
#define CB_EIO (-9)      /* a file could not be read or written, or is not in the expected format */

#define CB_HOST 0
#define CB_DEVICE 1

typedef struct cb_graph* cb_handle;

/*
 * Create a randomisation state from a CSR adjacency.
 *   n          number of nodes.
 *   row_ptr    n+1 int64 offsets, row_ptr[0] = 0, non-decreasing.
 *   col        row_ptr[n] int32 neighbour ids; every undirected edge {a,b}
 *              appears as b in row a and as a in row b; no self loops, no
 *              repeated neighbour (Section 2: simple graphs).  Rows need not
 *              be sorted.
 *   seed       64-bit seed of every random draw.
 *   first_step index of the first super step (0 normally; k to continue a
 *              chain exported after k super steps).
 *   mem_kind   where row_ptr and col live (CB_HOST / CB_DEVICE).
 *   cuda_stream a cudaStream_t to issue all work on, or NULL for a stream
 *              owned by the handle.
 *   out        receives the handle.
 * The inputs are copied; the caller keeps ownership of its buffers.  Returns
 * CB_EINVAL if the graph is not simple and symmetric.
 */
int cb_create(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
              uint64_t first_step, int mem_kind, void* cuda_stream, cb_handle* out);

/*
 * Create one state holding `count` independent graphs (an ensemble), each
 * randomised by its own chain exactly as cb_create would do for it alone:
 * graph i with its own seed; its node ids, permutation and shuffle keys are
 * local to it.  A super step (cb_global_trades) advances every graph by one
 * global trade in the same launches.  Section 3.3's odd-n rule holds per
 * graph: the node at a graph's last position is not traded.
 *   count      number of graphs, >= 1.
 *   n          host array of count node counts (n_i >= 0, sum < 2^31).
 *   row_ptr    the graphs' CSR offsets one after another: n_0+1 values for
 *              graph 0 (starting at 0), then n_1+1 for graph 1, ...
 *   col        the graphs' neighbour ids one after another (row_ptr_i[n_i]
 *              local ids in [0, n_i) for graph i); each graph simple and
 *              symmetric as for cb_create.
 *   seeds      host array of count seeds.
 *   first_step index of the first super step, shared by every graph.
 *   mem_kind   where row_ptr and col live; n and seeds are host arrays.
 *   cuda_stream, out as for cb_create.
 * Synchronises.  cb_info reports the totals (n counts one padding node per
 * odd graph); cb_graph_info each graph.
 */
int cb_create_batch(int32_t count, const int64_t* n, const int64_t* row_ptr, const int32_t* col,
                    const uint64_t* seeds, uint64_t first_step, int mem_kind, void* cuda_stream,
                    cb_handle* out);

/* Number of graphs of the handle (1 for cb_create); negative on error. */
int cb_graph_count(cb_handle h);

/* Nodes and undirected edges of graph `index` of the handle. */
int cb_graph_info(cb_handle h, int32_t index, int64_t* n, int64_t* m);

/*
 * Export graph `index` of the handle as its canonical edge list (local ids,
 * same format and rules as cb_export_edges).  Exporting several graphs after
 * the same super step computes the edge lists once.  Synchronises.
 */
int cb_export_graph(cb_handle h, int32_t index, int32_t* edges, int64_t capacity_pairs, int64_t* m_out,
                    int mem_kind);

/*
 * Run `supersteps` global trades (Def. "Undirected Global Trade").
 * Super step g (g counts from first_step):
 *   - permutation: node x gets key philox64(seed; x, 0, g, 0), nodes are
 *     sorted by (key, x); trade t is (order[2t], order[2t+1]); for odd n the
 *     node at the last position is not traded;
 *   - shuffle of trade t: each disjoint neighbour is keyed by its edge to u or
 *     v, identified by the positions lo < hi of the edge's endpoints at the
 *     start of super step g: Philox4x32-10(seed; lo, hi, g, 1) = r0..r3, key
 *     r0<<32|r1 if position lo belongs to trade t, else r2<<32|r3; D is
 *     ordered by (key, lo, hi) and u receives the first |A_{u-v}| elements.
 * philox64(...) = r0<<32 | r1 of Philox4x32-10 (Salmon et al., SC'11) with
 * key words (low, high) 32 bits of the seed.  Asynchronous on the handle's
 * stream (with the "timing" option on, a super step waits for the events of
 * the step two before it, so the host stays at most two steps ahead).
 * Returns CB_ERANGE if the step counter would pass 2^32 - 2.
 */
int cb_global_trades(cb_handle h, uint32_t supersteps);

/*
 * Export the current graph as its canonical edge list: m pairs [a, b] with
 * a < b in lexicographic order (Section 2 "ordered edges"), written as 2m
 * int32 values a0, b0, a1, b1, ... into `edges` (mem_kind says where).
 * edges == NULL: only *m_out is set.  capacity_pairs < m: CB_ESIZE and *m_out
 * is set.  For a handle of several graphs: every graph's list in turn, local
 * ids, m = the total.  Synchronises the handle's stream.
 */
int cb_export_edges(cb_handle h, int32_t* edges, int64_t capacity_pairs, int64_t* m_out,
                    int mem_kind);

/* Release every device buffer of the handle; NULL is ignored. */
void cb_destroy(cb_handle h);

/* Index of the next super step to run (first_step + super steps done). */
int cb_step(cb_handle h, uint64_t* g);

/* Wait for all work on the handle's stream; returns a latched device error. */
int cb_sync(cb_handle h);

/* Description of the last error on this handle ("" if none; NULL handle: global). */
const char* cb_last_error(cb_handle h);

/* Number of nodes and undirected edges (over every graph of the handle). */
int cb_info(cb_handle h, int64_t* n, int64_t* m);

/*
 * The permutation pi of super step g (Def. "Undirected Global Trade"):
 * order_out[p] = node at position p (n int32, mem_kind says where).  Does not
 * change the state.  For several graphs: each graph's permutation at step g
 * over its own range of the handle's node ids.  Synchronises the handle's
 * stream.
 */
int cb_permutation(cb_handle h, uint64_t g, int32_t* order_out, int mem_kind);

/*
 * Counters of the last cb_global_trades call, for tests and tuning
 * (synchronises the handle's stream; out[5] counts the kernels inside the
 * CUDA graphs replayed when "cuda_graph" is on):
 * out[0] = threshold passes of the last super step that ran trades: the
 *          first pass, each retry pass with deferred trades left, and the
 *          in-order pass when trades were still deferred,
 * out[1] = trades the first pass deferred,
 * out[2] = trades of the first pass on warps or parts of a warp (size
 *          classes 0..2), out[3] = on the larger teams (classes 3..8),
 * out[4] = trades whose workspace did not fit in shared memory,
 * out[5] = kernel launches issued by the last cb_global_trades or
 *          cb_uniform_trades call,
 * out[6] = trades still deferred after the retry passes (run by the in-order
 *          pass),
 * out[7 + k], k < 9 = trades of size class k in the first pass,
 * out[16 + k] = their directed entries (deg u + deg v summed).
 * `count` = capacity of out (at most 25 are written); returns the number of
 * counters written.
 */
int cb_stats(cb_handle h, int64_t* out, int count);

/*
 * Device time in milliseconds of the phases of the last cb_global_trades
 * call, summed over its super steps, measured with CUDA events on the
 * handle's stream while the "timing" option is on (zeros otherwise):
 * ms[0] = permutation of the next step and its row offsets, ms[1] = the
 * threshold phase (every trade's |A_{u-v}|-th smallest key, including the
 * passes that resolve dependent trades), ms[2] = the rebuild phase (new rows
 * for the next step), ms[3] = whole super steps, ms[4 + k], k < 9 = the
 * first threshold pass's kernel of size class k (0 where the class shares
 * another class's kernel), ms[13] = the retry passes over deferred trades,
 * ms[14] = the in-order pass.  Returns the number of values written
 * (<= count, at most 15).  Waits for the events still outstanding.
 */
int cb_timings(cb_handle h, double* ms, int count);

/*
 * Tuning / test knobs (key, value); returns CB_EINVAL for an unknown key or a
 * value out of range.  None changes any result.  Trade size = deg u + deg v.
 *   "cuda_graph" 1: record one super step (per ping-pong parity) as a CUDA
 *               graph on the first cb_global_trades call and replay it, one
 *               graph launch per super step [0].  Not while "timing" is on.
 *               The handle's stream must support capture (not the legacy
 *               default stream).  Changing any other option re-records.
 *   "tile_max"  trades up to this size run on warps or parts of a warp
 *               [128]; 0..128.
 *   "tile_paths" 1: trades up to tile_max entries run on warps or parts of
 *               a warp (see "lane_teams"); 0: on the larger teams [1].
 *   "block_max" trades up to this size run on a 256-thread CTA [1024];
 *               0..2048 (values below tile_max act as tile_max).
 *   "smem_max"  larger trades run on a 1024-thread CTA; with "cta_paths" 1
 *               up to min(4096, smem_max) entries in registers, with 0 up
 *               to smem_max entries in shared memory; more in a
 *               global-memory workspace [8192]; 64..8192.
 *   "cta_paths" 1: threshold phase of the 256- and 1024-thread classes with
 *               the entries in registers (4 per thread); 0: in shared
 *               memory [1].
 *   "cand_max"  register paths: when at most this many elements share the
 *               threshold's leading key bits they are ranked directly,
 *               else more radix digits follow [32]; 1..32 (a test knob).
 *   "inorder_threads" CTA size of the pass that runs deferred trades in
 *               index order: 1024 (large trades in shared memory) or 256
 *               (four CTAs per SM; trades above block_max from global
 *               memory) [1024; 256 for cb_create_batch].
 *   "uniform_threads" CTA size of the executor of cb_uniform_trades: 256
 *               (two CTAs per SM), 512 or 1024 (more threads per hub trade,
 *               fewer trades at once) [1024].
 *   "lane_teams" 1: trades of at most 32 / 64 entries run on teams of 8 /
 *               16 lanes, several per warp; 0: on whole warps [1].
 *   "retry_passes" parallel passes over the deferred trades between the
 *               first pass and the in-order pass, each running every deferred
 *               trade whose dependencies have published by then [2]; 0..4.
 *   "relaxed"   1: relaxed global trades (Def. "Relaxed global trade",
 *               Appendix EM-GCB): super step g orders the nodes by
 *               h(x) = (a x + b) mod p, p the smallest prime >= n, with
 *               a = 1 + (philox64(seed; 0, 0, g, 4) mod (p - 1)) and b =
 *               (r2<<32|r3 of the same call) mod p, computed without a sort;
 *               0: the Philox key sort [0].  May be switched between super
 *               steps (the current step is laid out again).  Handles of one
 *               graph only (CB_EINVAL for cb_create_batch).
 *   "wide_pack" 1: the rebuild reads 16-byte far-trade records even when
 *               n <= 2^29 would allow 8-byte ones (a test knob) [0].
 *   "bucket_cap" largest permutation bucket sorted in shared memory [2048];
 *               larger buckets take the global-memory fallback; 2..4096.
 *   "timing"    1: record CUDA events around the phases and the first
 *               pass's kernels of each super step, in two sets used in turn
 *               (the host waits for a set two steps after recording it) [0].
 *   "wait_ms"   longest single device wait, in milliseconds [1000 for a
 *               super step, 20000 for uniform trades]; 1..600000.  A wait
 *               that runs out makes the call (or the next cb_sync) return
 *               CB_ETIMEOUT.
 *   "hold_publish" 1: trades never publish that their threshold is ready,
 *               so a trade that depends on another waits until "wait_ms"
 *               runs out (a test of the timeout path) [0].
 *   "hold_trade" uniform trades: messages to this trade (index within the
 *               call) are dropped, so it never runs and the executor's
 *               waits run out (a test of the timeout path); -1: none [-1].
 *   "presence"  T > 0: record the edge presence of every node pair of every
 *               graph now and after each of the next T super steps (for
 *               cb_autocorr; one bit per pair and state, T <= 10^6, at most
 *               64 GB); super steps then run without the recorded CUDA
 *               graphs, plus one recording kernel each.  Setting it again
 *               starts a new record; 0 stops and frees it [0].
 *   "fix_passes" passes of the rebuild over slices of the far trades (0:
 *               as many as keep one slice's records in L2) [0]; 0..64.
 *   "swap_stats" 1: count neighbourhood swaps (see cb_swap_counts) from zero
 *               in every later super step and uniform trade; super steps
 *               then run without the recorded CUDA graphs, plus one counting
 *               kernel each.  0: stop counting [0].  Handles of one graph
 *               only (CB_EINVAL for cb_create_batch).
 */
int cb_set_option(cb_handle h, const char* key, int64_t value);

/*
 * Swap counts since "swap_stats" was last set to 1 (Appendix "Swaps
 * performed by Curveball and Global Curveball").
 *   - A trade of u and v performs as many neighbourhood swaps as edge ends
 *     that change node: twice the pairs of disjoint neighbours it exchanges.
 *     Fig. 2's sigma exchanges four edges.
 *   - deg(u) + deg(v) swaps are possible.
 *   - For odd n the untraded node of a global trade counts in neither.
 * *performed / *possible is the fraction the appendix plots.  Both are 0
 * when counting was never on.  Synchronises the handle's stream.
 */
int cb_swap_counts(cb_handle h, int64_t* performed, int64_t* possible);

/*
 * Edge autocorrelation of the recorded chain (Section 5.1, "Mixing of
 * Edge-Switching, Curveball and Global Curveball").  For every node pair
 * that is an edge in at least one recorded state (option "presence"), the
 * series Z_t (edge present in state t) is thinned to every k-th entry, and
 * the transitions of the thinned series are fitted to an independent and to
 * a first-order Markov model; the edge counts as correlated when the Markov
 * model fits better by the Bayesian information criterion:
 * G^2 = 2 (L_Markov - L_independent) > ln N, N the number of thinned
 * transitions.  (The paper cites the criterion without printing it; this is
 * the reading used here.)  A constant series, or one with N < 2, counts as
 * independent.
 *   graph       graph index of a batch handle, or -1 for all graphs.
 *   kmax        thinnings k = 1..kmax, 1 <= kmax <= 64.
 *   correlated  kmax host int64: edges classified as correlated for each k.
 *   near_ties   kmax host int64 (may be NULL): decisions with
 *               |G^2 - ln N| < 1e-9, which rounding could flip.
 *   occurring   (may be NULL) edges that occur in some recorded state.
 *   states      (may be NULL) recorded states (1 + super steps recorded).
 * The fraction of correlated edges is correlated[k-1] / *occurring.
 * Synchronises the handle's stream.
 */
int cb_autocorr(cb_handle h, int32_t graph, int32_t kmax, int64_t* correlated, int64_t* near_ties,
                int64_t* occurring, int64_t* states);

/*
 * The permutation of super step g for n nodes and `seed` (the same order as
 * cb_permutation), computed without allocating anything.  The paper has no
 * counterpart: this serves callers that may not allocate device memory
 * themselves, such as code running inside a host framework that owns every
 * device allocation, or a latency-critical loop where cudaMalloc could
 * synchronise the device or fail.
 *   n          number of nodes, 0 <= n <= 2^20 (larger n: CB_ESIZE).
 *   seed, g    as in cb_global_trades; g < 2^32 - 2.
 *   order_out  n int32 in device memory (caller-owned): order_out[p] = node
 *              at position p.
 *   cuda_stream the cudaStream_t to run on (NULL: the default stream); the
 *              call returns without waiting for the result.
 * Scratch: one static 13 MiB device array, held by every device that loads
 * the library until the process exits, and shared by every call on that
 * device.  The first call on a device looks up that array's device address
 * (once per device, with the device current) and keeps it for the life of
 * the process; make the first call before any stream capture.  Resetting a
 * device (cudaDeviceReset) after that call is not supported: the kept
 * address would no longer name the array.  Each call clears the counters it needs, but calls that
 * overlap on the GPU (different streams, or host threads) race on the shared
 * scratch and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * other allocating routine is called.  Errors are reported through
 * cb_last_error(NULL).
 */
int cb_permutation_static(int64_t n, uint64_t seed, uint64_t g, int32_t* order_out, void* cuda_stream);

/*
 * Pick the fastest work split for this handle: runs up to max_steps real
 * super steps (they advance the chain; the result does not depend on the
 * options): one to load the kernels, then the rest shared evenly by the
 * current settings and the candidate settings, one knob at a time, of
 * "tile_max", "block_max", "smem_max", "inorder_threads" and
 * "retry_passes", timed with CUDA events; a candidate replaces the best
 * setting so far only when it is at least 2 % faster.  chosen (may be NULL) receives up to
 * `count` values: tile_max, block_max, smem_max, inorder_threads, super
 * steps used, retry_passes.  Returns the number of values written.
 */
int cb_autotune(cb_handle h, uint32_t max_steps, int64_t* chosen, int count);

/*
 * cb_autotune with a file cache.  The key (cb_tune_key) names the GPU (device
 * name, SM count), floor(log2 n), floor(log2 graphs) and the handle's degree
 * distribution: for each degree bit length b = 0..32, the share of directed
 * entries of the nodes whose degree has b bits, in 64ths.  When cache_path
 * holds the key, its settings are applied (no super step runs; chosen[4] =
 * 0); otherwise cb_autotune runs and its choice is stored under the key.  The
 * cache is a JSON file, {"version": 1, "entries": [{"key": ..., "tile_max":
 * ..., "block_max": ..., "smem_max": ..., "inorder_threads": ...,
 * "retry_passes": ...}, ...]}, written whole to cache_path + ".tmp" and
 * renamed over cache_path.  chosen / count and the return value as for
 * cb_autotune; CB_EIO when the file cannot be read or written or is not such
 * a cache (it is then left unchanged).
 */
int cb_autotune_cached(cb_handle h, uint32_t max_steps, const char* cache_path, int64_t* chosen, int count);

/*
 * The cache key of a handle (see cb_autotune_cached) into key[0..cap), NUL
 * terminated.  Runs one histogram kernel over the degrees and synchronises the
 * handle's stream.  Returns the key's length, CB_ESIZE if cap is too small.
 */
int cb_tune_key(cb_handle h, char* key, int cap);

/*
 * Host-only access to a tuning cache file (no device work).  lookup: the
 * settings stored under key into vals (tile_max, block_max, smem_max,
 * inorder_threads, retry_passes; up to count of them); returns how many were
 * written, 0 when the file or the key does not exist.  store: vals (exactly 5,
 * in that order) under key, replacing an entry with the same key and keeping
 * the others.  A key may not contain '"', '\', '{', '}' or control
 * characters (CB_EINVAL).  Both return CB_EIO for a file that cannot be read
 * or written or is not a tuning cache.
 */
int cb_tune_cache_lookup(const char* path, const char* key, int64_t* vals, int count);
int cb_tune_cache_store(const char* path, const char* key, const int64_t* vals, int count);

#ifdef __cplusplus
}
#endif

#endif /* CB_H */
