/*
 * cb_serve.h -- serving loop of libcb.so: randomisation requests of different
 * sizes admitted while a device-memory budget allows, kept resident on the
 * device and stepped together (continuous batching).
 *
 * A request is one graph (CSR, as for cb_create), a seed and a number of
 * global Curveball super steps (Def. "Undirected Global Trade", Section 3.3);
 * its result is the canonical edge list after those super steps, identical
 * to what cb_create + cb_global_trades + cb_export_edges give for the same
 * graph and seed alone.  The paper has no serving layer; this is the systems
 * wrapper around the super step.
 *
 * The server runs two host threads of its own:
 *   - the admitter takes queued requests in arrival order while the estimated
 *     device bytes of the resident ones (cb_estimate_bytes) stay within the
 *     budget and fewer than max_active are resident, creates each one's state
 *     on a stream of its own (stream-ordered device memory, CUDA-graph super
 *     step), and, for finished requests, exports the edge list to host memory
 *     and releases the device memory;
 *   - the stepper issues one super step of every resident request in turn, at
 *     most `depth` super steps in flight per request, so the super steps of
 *     all resident requests overlap on the device and a request that arrives
 *     while others run starts as soon as a slot and memory are free.
 * A request larger than the whole budget fails (CB_ENOMEM in its result).
 * Times are seconds on the host's monotonic clock since the server started.
 * Every call is thread-safe.
 */
#ifndef CB_SERVE_H
#define CB_SERVE_H

#include <stdint.h>

#include "cb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cb_server* cb_server_t;

/*
 * Start a server on the current CUDA device.
 *   hbm_budget_bytes  device bytes the resident requests may take together.
 *   max_active        most requests resident at once (>= 1).
 *   depth             super steps in flight per request (1..8).
 */
int cb_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t depth, cb_server_t* out);

/*
 * Queue a request.  row_ptr (n+1 int64) and col (row_ptr[n] int32) are host
 * memory and are copied before the call returns.  *id receives the request
 * id (0, 1, 2, ... in submission order).
 */
int cb_server_submit(cb_server_t s, int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                     uint32_t supersteps, int64_t* id);

/*
 * Ids of requests finished (successfully or not) since the last call, at
 * most `capacity`; waits up to timeout_ms for one when none is ready.
 * Returns the number written.
 */
int cb_server_poll(cb_server_t s, int64_t* ids, int32_t capacity, int32_t timeout_ms);

/*
 * Result of finished request `id`: *m_out edges as 2m int32 (host memory,
 * canonical order) into `edges` (NULL: size query, the request is kept).
 * times (may be NULL) receives 4 values: submitted, admitted (memory
 * reserved), resident (state created on the device), finished (edges on the
 * host).  With `edges` given the request is released afterwards.  Returns
 * the request's own error code if it failed (message in cb_last_error(NULL)).
 */
int cb_server_result(cb_server_t s, int64_t id, int32_t* edges, int64_t capacity_pairs, int64_t* m_out,
                     double* times);

/*
 * Counters: out[0] submitted, [1] queued, [2] resident, [3] finished,
 * [4] estimated device bytes reserved now, [5] the peak of [4],
 * [6] super steps issued, [7] failed requests.  Returns the number written.
 */
int cb_server_stats(cb_server_t s, int64_t* out, int32_t count);

/* Stop both threads (requests still queued or resident are dropped) and free everything. */
void cb_server_destroy(cb_server_t s);

/*
 * Device bytes a state of n nodes, nnz directed entries (row_ptr[n]) and
 * largest degree max_degree takes at most, including the temporary buffer
 * of a host export: the admission estimate.
 */
int64_t cb_estimate_bytes(int64_t n, int64_t nnz, int64_t max_degree);

/* Device bytes the handle holds now and at most so far. */
int cb_device_bytes(cb_handle h, int64_t* now, int64_t* peak);

#ifdef __cplusplus
}
#endif

#endif /* CB_SERVE_H */
