// The C ABI declared in include/cb.h: handle lifetime, input import and
// validation, the super-step loop and the canonical export.
#include <algorithm>
#include <cstring>
#include <string>

#include "cb_internal.cuh"

namespace cb {

size_t trade_ws_slice_bytes(int64_t max_trade);

namespace {
thread_local std::string g_error;

__global__ void k_degrees(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ deg,
                          unsigned long long* __restrict__ maxdeg) {
  unsigned long long local = 0;
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = rp[x + 1] - rp[x];
    deg[x] = static_cast<int32_t>(d);
    if (d > 0 && static_cast<unsigned long long>(d) > local) local = static_cast<unsigned long long>(d);
  }
  atomicMax(maxdeg, local);
}

__global__ void k_gather_deg(int64_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ deg_id,
                             int32_t* __restrict__ out) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x)
    out[p] = deg_id[order[p]];
}

unsigned grid1d(int64_t work, int num_sms) {
  const int64_t want = (work + 255) / 256;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(num_sms) * 16)));
}

// Spare entries after each adjacency buffer: a bulk copy of a trade's row
// range moves whole 16-byte units and may read up to 3 entries past the end.
constexpr int64_t kColPad = 16;

// Device memory of a handle is stream-ordered (the device's memory pool, on
// the handle's stream): creating and destroying handles never waits for work
// of other streams, so many handles can come and go while others run.
cudaError_t dmalloc(Graph* h, void** p, size_t bytes) {
  const cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e == cudaSuccess) {
    h->dev_bytes += static_cast<int64_t>(bytes);
    h->dev_bytes_peak = std::max(h->dev_bytes_peak, h->dev_bytes);
  }
  return e;
}
template <class T>
cudaError_t dalloc(Graph* h, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  return dmalloc(h, reinterpret_cast<void**>(p), sizeof(T) * static_cast<size_t>(count));
}
void dfree(Graph* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

void release(Graph* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_uniform(h);
  free_presence(h);
  void* bufs[] = {h->deg_id, h->rp_id, h->order[0], h->order[1], h->rp[0], h->rp[1], h->col[0], h->col[1],
                  h->pos_next, h->M, h->deg_next, h->stash, h->thr_key, h->thr_tb, h->thr_top, h->done,
                  h->lists, h->dlist, h->Minv, h->cls_flag, h->cls_scan,
                  h->counters, h->err,
                  h->ws_global, h->sort_ws, h->scan_ws, h->segs, h->seg_of, h->pairs, h->far_pack,
                  h->lcg_ab, h->lcg_gaps, h->swaps};
  if (h->stream)
    for (void* b : bufs) dfree(h, b);
  for (auto& x : h->step_exec)
    if (x) cudaGraphExecDestroy(x);
  delete[] h->hsegs;
  delete[] h->host_counters;
  for (auto& set : h->ev)
    for (auto& e : set)
      if (e) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Read the latched device error word; synchronises the stream.
int read_device_error(Graph* h) {
  int32_t e = 0;
  CB_CUDA(h, cudaMemcpyAsync(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (e != kErrNone) {
    if (is_timeout(e)) {
      h->latched = CB_ETIMEOUT;
      return fail(h, CB_ETIMEOUT, "a bounded device wait ran out (code " + std::to_string(e) + ")");
    }
    h->latched = CB_ECHECK;
    return fail(h, CB_ECHECK, "device check failed (code " + std::to_string(e) + ")");
  }
  return CB_OK;
}

int size_trade_workspace(Graph* h) {
  if (h->ws_global) {
    dfree(h, h->ws_global);
    h->dev_bytes -= static_cast<int64_t>(h->ws_slice * h->ws_ctas);
    h->ws_global = nullptr;
  }
  // a slice per CTA for trades whose workspace is not in shared memory: above
  // smem_max on the 1024-thread path, above block_max in the in-order pass
  const int64_t max_trade = 2 * h->maxdeg;
  const int64_t block_max = std::max(h->block_max, std::min(h->tile_max, kTileMaxCap));
  h->ws_ctas = h->num_sms * 4;
  h->ws_slice = 0;
  if (max_trade > std::min<int64_t>(h->smem_max, block_max) || h->maxdeg > 16384) {
    h->ws_slice = trade_ws_slice_bytes(std::max<int64_t>(max_trade, 1));
    const size_t budget = size_t(2) << 30;
    h->ws_ctas = static_cast<int>(std::max<size_t>(1, std::min<size_t>(h->num_sms * 4, budget / h->ws_slice)));
    CB_CUDA(h, dmalloc(h, &h->ws_global, h->ws_slice * h->ws_ctas));
  }
  return CB_OK;
}

}  // namespace

int check_device_error(Graph* h) { return read_device_error(h); }

cudaError_t dev_alloc(Graph* h, void** p, size_t bytes) { return dmalloc(h, p, bytes); }

int fail(Graph* g, int code, const std::string& msg) {
  if (g) g->last_error = msg;
  else g_error = msg;
  return code;
}

int cuda_fail(Graph* g, cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? CB_ENOMEM : CB_ECUDA;
  cudaGetLastError();  // clear a non-sticky error
  return fail(g, code, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace cb

namespace cb {
namespace {

// Batch input: graph i's offsets start at rp_in + rpo[i] (n_i + 1 values, the
// first 0) and its entries, local ids, sit at the same entry offsets in col
// (padding nodes have no entries).  Builds the combined id-space offsets and
// adds each graph's first node id to its entries.
__global__ void k_batch_offsets(int64_t N, const Seg* __restrict__ segs, const int32_t* __restrict__ seg_of,
                                const int64_t* __restrict__ rp_in, const int64_t* __restrict__ rpo,
                                const int64_t* __restrict__ eoff, int64_t nnz, int64_t* __restrict__ rp,
                                int32_t* err) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x <= N; x += int64_t(gridDim.x) * blockDim.x) {
    if (x == N) {
      rp[N] = nnz;
      continue;
    }
    const int i = seg_of[x];
    const int64_t l = x - segs[i].off, n = segs[i].n;
    const int64_t v = rp_in[rpo[i] + (l < n ? l : n)];
    if (l == 0 && v != 0) atomicCAS(err, 0, static_cast<int32_t>(kErrValidate));
    rp[x] = eoff[i] + v;
  }
}

__global__ void k_batch_cols(int64_t N, const Seg* __restrict__ segs, const int32_t* __restrict__ seg_of,
                             const int64_t* __restrict__ rp, int32_t* __restrict__ col, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < N; x += nw) {
    const Seg& S = segs[seg_of[x]];
    const int32_t off = static_cast<int32_t>(S.off), n = static_cast<int32_t>(S.n);
    for (int64_t e = rp[x] + lane; e < rp[x + 1]; e += 32) {
      const int32_t y = col[e];
      if (y < 0 || y >= n) atomicCAS(err, 0, static_cast<int32_t>(kErrValidate));
      col[e] = y + off;
    }
  }
}

__global__ void k_fill_seg_of(int64_t N, const Seg* __restrict__ segs, int nseg, int32_t* __restrict__ seg_of) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < N; x += int64_t(gridDim.x) * blockDim.x) {
    int lo = 0, hi = nseg;   // last segment with off <= x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (segs[mid].off <= x) lo = mid; else hi = mid;
    }
    seg_of[x] = lo;
  }
}

Graph* new_graph(void* cuda_stream, int* rc) {
  *rc = CB_OK;
  cb_graph* h = new (std::nothrow) cb_graph();
  if (!h) {
    *rc = fail(nullptr, CB_ENOMEM, "host allocation failed");
    return nullptr;
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
      h->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    *rc = cuda_fail(nullptr, e, "device set-up");
    delete h;
    return nullptr;
  }
  return h;
}

void destroy_graph(Graph* h) {
  release(h);
  delete static_cast<cb_graph*>(h);
}

// Scratch int32: the trade classes' counts per 2048-trade chunk, then
// (rebuild) the first row of each 2048-entry chunk plus one.
int64_t cls_flag_count(int64_t ntasks, int64_t nnz) {
  return std::max<int64_t>(kClasses * (ntasks / 2048 + 1), nnz / 2048 + 2);
}
// Scratch int64: the exclusive scan of those counts.
int64_t cls_scan_count(int64_t ntasks) { return kClasses * (ntasks / 2048 + 1) + 1; }

// Common part of handle creation.  On entry: n, nnz, the segment table (host
// and device, seg_of for batches) and the id-space CSR (rp_id, col[0],
// unsorted rows) are in place.  Validates, sizes the workspaces and lays the
// graph out for its first super step.
int finish_create(Graph* h) {
  const int64_t n = h->n, nnz = h->nnz;
  cudaStream_t s = h->stream;
  int rc;
  h->m = nnz / 2;
  h->T = n / 2;
  h->ntasks = h->T + (n & 1);
  if ((rc = init_trade_kernels(h)) || (rc = init_perm_kernels(h))) return rc;
  if ((rc = check_row_offsets(h, h->rp_id, n))) return rc;
  {
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(h->counters);
    CB_CUDA(h, cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
    if (n) k_degrees<<<grid1d(n, h->num_sms), 256, 0, s>>>(n, h->rp_id, h->deg_id, dmax);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    unsigned long long hm = 0;
    CB_CUDA(h, cudaMemcpyAsync(&hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, s));
    if ((rc = check_device_error(h))) {
      h->last_error = "row_ptr is not a valid CSR offset array (degrees in [0, n), ids in range)";
      return CB_EINVAL;
    }
    h->maxdeg = static_cast<int64_t>(hm);
  }
  h->sort_ws_bytes = perm_ws_bytes(std::max<int64_t>(n, 1), h->nbuckets);
  h->scan_ws_bytes = scan_ws_bytes(std::max<int64_t>(n + 1, h->nbuckets + 1));
  if (dalloc(h, &h->order[0], n) || dalloc(h, &h->order[1], n) || dalloc(h, &h->rp[0], n + 1) || dalloc(h, &h->rp[1], n + 1) ||
      dalloc(h, &h->pos_next, n) || dalloc(h, &h->M, n) || dalloc(h, &h->Minv, n) || dalloc(h, &h->deg_next, n) ||
      dalloc(h, &h->stash, nnz) ||
      dalloc(h, &h->thr_key, h->ntasks) || dalloc(h, &h->thr_tb, h->ntasks) || dalloc(h, &h->done, h->ntasks) ||
      dalloc(h, &h->far_pack, h->ntasks) ||
      dalloc(h, &h->thr_top, h->ntasks) || dalloc(h, &h->lists, h->ntasks) || dalloc(h, &h->dlist, 2 * h->ntasks) ||
      dalloc(h, &h->cls_flag, cls_flag_count(h->ntasks, nnz)) || dalloc(h, &h->cls_scan, cls_scan_count(h->ntasks)) ||
      dmalloc(h, &h->sort_ws, h->sort_ws_bytes) || dmalloc(h, &h->scan_ws, h->scan_ws_bytes))
    return fail(h, CB_ENOMEM, "device allocation failed");
  CB_CUDA(h, cudaMemsetAsync(h->done, 0, sizeof(uint32_t) * std::max<int64_t>(h->ntasks, 1), s));
  // the rebuild reads 8 placeholders (32 B) and 8 side words (16 B) per vector load
  if ((reinterpret_cast<uintptr_t>(h->col[0]) | reinterpret_cast<uintptr_t>(h->col[1])) % 16 ||
      reinterpret_cast<uintptr_t>(h->stash) % 16)
    return fail(h, CB_ECUDA, "device allocation not aligned for vector loads");
  if ((rc = size_trade_workspace(h))) return rc;
  // rows in id space, sorted (sorted input is used as it is), then validated:
  // simple and symmetric
  bool sorted = false;
  if ((rc = rows_sorted(h, h->rp_id, h->col[0], n, &sorted))) return rc;
  int32_t* idcol = h->col[0];
  if (!sorted) {
    if ((rc = permute_rows(h, n, h->rp_id, h->col[0], nullptr, nullptr, h->rp_id, h->col[1]))) return rc;
    idcol = h->col[1];
  }
  if ((rc = validate_sorted_graph(h, h->rp_id, idcol, n, idcol == h->col[0] ? h->col[1] : h->col[0]))) return rc;
  if ((rc = check_device_error(h))) {
    h->last_error = "graph is not simple and symmetric";
    return CB_EINVAL;
  }
  // position-space layout of the first super step (rows are sets: no sort);
  // the step's adjacency lives in col[cur = 0]
  h->cur = 0;
  if ((rc = compute_permutation(h, 0, -1, h->order[0], h->pos_next))) return rc;
  if (n) k_gather_deg<<<grid1d(n, h->num_sms), 256, 0, s>>>(n, h->order[0], h->deg_id, h->deg_next);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(h->deg_next, h->rp[0], n, h->scan_ws, s, &h->launches));
  int32_t* pcol = idcol == h->col[0] ? h->col[1] : h->col[0];
  if ((rc = relabel_rows(h, n, h->rp_id, idcol, h->order[0], h->pos_next, h->rp[0], pcol))) return rc;
  if (pcol != h->col[0]) std::swap(h->col[0], h->col[1]);
  return check_device_error(h);
}

void drop_graphs(Graph* h) {
  for (auto& x : h->step_exec)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
}

// Records one super step per ping-pong parity into a CUDA graph.  A super
// step has no host round trip and reads every per-step value (step counters,
// counts) from device memory, so replaying the two graphs alternately is the
// same as calling super_step.  Host state is left as it was.
int capture_step_graphs(Graph* h) {
  const int cur0 = h->cur;
  const uint64_t g0 = h->g;
  const int64_t l0 = h->launches;
  // a super step leaves its output in the buffer it read (col[cur] before
  // and after), so parity p is recorded with that buffer as col[p]
  int32_t* const adj = h->col[cur0];
  int32_t* const spare = h->col[1 - cur0];
  int rc = CB_OK;
  for (int p = 0; p < 2 && rc == CB_OK; ++p) {
    h->cur = p;
    h->col[p] = adj;
    h->col[1 - p] = spare;
    const int64_t lb = h->launches;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      rc = cuda_fail(h, e, "cudaStreamBeginCapture");
      break;
    }
    rc = super_step(h);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(h->stream, &gr);
    h->step_launches = h->launches - lb;
    if (rc == CB_OK && e != cudaSuccess) rc = cuda_fail(h, e, "cudaStreamEndCapture");
    if (rc == CB_OK) {
      e = cudaGraphInstantiate(&h->step_exec[p], gr, 0);
      if (e != cudaSuccess) rc = cuda_fail(h, e, "cudaGraphInstantiate");
    }
    if (gr) cudaGraphDestroy(gr);
    h->cur = cur0;
    h->g = g0;
  }
  h->col[cur0] = adj;
  h->col[1 - cur0] = spare;
  h->launches = l0;
  if (rc) drop_step_graphs(h);
  return rc;
}

// Every graph's canonical pairs (local ids) of the current step in h->pairs.
int ensure_pairs(Graph* h) {
  if (h->pairs && h->pairs_step == h->g) return CB_OK;
  if (!h->pairs && dalloc(h, &h->pairs, 2 * std::max<int64_t>(h->m, 1)))
    return fail(h, CB_ENOMEM, "device allocation failed");
  int rc;
  if ((rc = export_sorted_pairs(h, h->pairs))) return rc;
  if ((rc = check_device_error(h))) return rc;
  h->pairs_step = h->g;
  return CB_OK;
}

int copy_pairs(Graph* h, int64_t first, int64_t count, int32_t* edges, int mem_kind) {
  if (count == 0) return CB_OK;
  CB_CUDA(h, cudaMemcpyAsync(edges, h->pairs + 2 * first, sizeof(int32_t) * 2 * count,
                             mem_kind == CB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  return CB_OK;
}

uint64_t next_prime_host(uint64_t n) {
  for (uint64_t p = n < 2 ? 2 : n;; ++p) {
    bool prime = true;
    for (uint64_t d = 2; d * d <= p; ++d)
      if (p % d == 0) {
        prime = false;
        break;
      }
    if (prime) return p;
  }
}

// Switch between permutations by Philox key sort and by a linear congruential
// map (Def. "Relaxed global trade") between super steps: the current graph is
// taken back to node-id rows, the current step's permutation is drawn in the
// new mode, and the rows are laid out again.  The chain state is the graph
// and the step index, so the switch is seamless.
int set_relaxed(Graph* h, bool on) {
  if (h->nseg != 1) return fail(h, CB_EINVAL, "relaxed permutations are for handles of one graph");
  if (on == h->relaxed) return CB_OK;
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  int rc;
  if (on && !h->lcg_ab) {
    h->lcg_p = next_prime_host(static_cast<uint64_t>(std::max<int64_t>(n, 2)));
    if (h->lcg_p - static_cast<uint64_t>(n) >= static_cast<uint64_t>(kMaxLcgGaps))
      return fail(h, CB_EINVAL, "prime gap above the relaxed permutation's limit");
    if (dalloc(h, &h->lcg_ab, 2) || dalloc(h, &h->lcg_gaps, kMaxLcgGaps + 1))
      return fail(h, CB_ENOMEM, "device allocation failed");
  }
  const int spare = 1 - h->cur;
  // node-id rows of the current graph into col[spare]
  if ((rc = invert_permutation(h, h->order[h->cur], h->pos_next))) return rc;
  if ((rc = permute_rows(h, n, h->rp[h->cur], h->col[h->cur], h->pos_next, h->order[h->cur], h->rp_id,
                         h->col[spare])))
    return rc;
  h->relaxed = on;
  if ((rc = compute_permutation(h, 0, -1, h->order[h->cur], h->pos_next))) return rc;
  if (n) k_gather_deg<<<grid1d(n, h->num_sms), 256, 0, s>>>(n, h->order[h->cur], h->deg_id, h->deg_next);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(h->deg_next, h->rp[h->cur], n, h->scan_ws, s, &h->launches));
  if ((rc = relabel_rows(h, n, h->rp_id, h->col[spare], h->order[h->cur], h->pos_next, h->rp[h->cur],
                         h->col[h->cur])))
    return rc;
  h->pairs_step = ~0ull;
  return check_device_error(h);
}

int upload_segs(Graph* h) {
  CB_CUDA(h, cudaMemcpyAsync(h->segs, h->hsegs, sizeof(Seg) * h->nseg, cudaMemcpyHostToDevice, h->stream));
  return CB_OK;
}

}  // namespace

int64_t estimate_handle_bytes(int64_t n, int64_t nnz, int64_t maxdeg, int num_sms) {
  // mirrors the allocations of cb_create + finish_create + size_trade_workspace
  // + a host export's temporary pairs (2m int32)
  const int64_t ntasks = n / 2 + (n & 1);
  const int64_t nb = int64_t(1) << bucket_bits(n);
  int64_t b = 0;
  b += sizeof(Seg) + 8 * (n + 1) + 4 * n + 2 * 4 * (nnz + kColPad) + 32 + 8 * kCounters;   // cb_create
  b += 2 * 4 * n + 2 * 8 * (n + 1) + 4 * 4 * n + 2 * nnz;                                 // per node, side words
  b += ntasks * (8 + 8 + 4 + 16 + 1 + 4 + 8) + 4 * cls_flag_count(ntasks, nnz) + 8 * cls_scan_count(ntasks) + 32;
  b += static_cast<int64_t>(perm_ws_bytes(std::max<int64_t>(n, 1), nb) + scan_ws_bytes(std::max(n + 1, nb + 1)));
  const int64_t max_trade = 2 * maxdeg;
  if (max_trade > kBlockMaxDefault || maxdeg > 16384) {   // default block_max
    const size_t slice = trade_ws_slice_bytes(std::max<int64_t>(max_trade, 1));
    const size_t ctas = std::max<size_t>(1, std::min<size_t>(num_sms * 4, (size_t(2) << 30) / slice));
    b += static_cast<int64_t>(slice * ctas);
  }
  b += 4 * std::max<int64_t>(nnz, 2);
  return b + b / 64 + (int64_t(16) << 20);   // pool rounding and per-allocation slack
}

int prepare_step_graphs(Graph* h) {
  if (!h->use_graph || h->step_exec[0]) return CB_OK;
  return capture_step_graphs(h);
}

void drop_step_graphs(Graph* h) { drop_graphs(h); }

}  // namespace cb

using namespace cb;

extern "C" {

int cb_create(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed, uint64_t first_step,
              int mem_kind, void* cuda_stream, cb_handle* out) {
  if (!out) return fail(nullptr, CB_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0 || n > 0x7fffffffLL || !row_ptr || (mem_kind != CB_HOST && mem_kind != CB_DEVICE))
    return fail(nullptr, CB_EINVAL, "bad n, row_ptr or mem_kind");
  if (first_step >= 0xfffffffeull) return fail(nullptr, CB_ERANGE, "first_step too large");
  int rc;
  Graph* h = new_graph(cuda_stream, &rc);
  if (!h) return rc;
  auto bail = [&](int code) {
    g_error = h->last_error;
    destroy_graph(h);
    return code;
  };
  const cudaMemcpyKind kind = mem_kind == CB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int64_t ends[2] = {0, 0};
  if (mem_kind == CB_HOST) {
    ends[0] = row_ptr[0];
    ends[1] = row_ptr[n];
  } else {
    if (cudaMemcpy(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(fail(h, CB_EINVAL, "row_ptr is not readable device memory"));
  }
  const int64_t nnz = ends[1];
  if (ends[0] != 0 || nnz < 0 || (nnz & 1) || nnz / 2 >= (int64_t(1) << 32) || (nnz > 0 && !col))
    return bail(fail(h, CB_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] even, < 2^33"));
  h->n = n;
  h->nnz = nnz;
  h->seed = seed;
  h->g = first_step;
  h->nseg = 1;
  h->hsegs = new (std::nothrow) Seg[1];
  if (!h->hsegs) return bail(fail(h, CB_ENOMEM, "host allocation failed"));
  {
    Seg& S = h->hsegs[0];
    S = Seg{};
    S.seed = seed;
    S.n = S.span = n;
    S.m = nnz / 2;
    S.g = static_cast<uint32_t>(first_step);
    S.B = bucket_bits(n);
    h->nbuckets = int64_t(1) << S.B;
  }
  cudaStream_t s = h->stream;
  if (dalloc(h, &h->segs, 1) || dalloc(h, &h->rp_id, n + 1) || dalloc(h, &h->deg_id, n) || dalloc(h, &h->col[0], nnz + kColPad) ||
      dalloc(h, &h->col[1], nnz + kColPad) || dalloc(h, &h->err, 8) || dalloc(h, &h->counters, kCounters) ||
      !(h->host_counters = new (std::nothrow) int64_t[kCounters]))
    return bail(fail(h, CB_ENOMEM, "device allocation failed"));
  CB_CUDA(h, cudaMemsetAsync(h->err, 0, 8 * sizeof(int32_t), s));
  if ((rc = upload_segs(h))) return bail(rc);
  CB_CUDA(h, cudaMemcpyAsync(h->rp_id, row_ptr, sizeof(int64_t) * (n + 1), kind, s));
  if (nnz) CB_CUDA(h, cudaMemcpyAsync(h->col[0], col, sizeof(int32_t) * nnz, kind, s));
  if ((rc = finish_create(h))) return bail(rc);
  *out = static_cast<cb_graph*>(h);
  return CB_OK;
}

int cb_create_batch(int32_t count, const int64_t* n, const int64_t* row_ptr, const int32_t* col,
                    const uint64_t* seeds, uint64_t first_step, int mem_kind, void* cuda_stream, cb_handle* out) {
  if (!out) return fail(nullptr, CB_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !n || !seeds || !row_ptr || (mem_kind != CB_HOST && mem_kind != CB_DEVICE))
    return fail(nullptr, CB_EINVAL, "bad count, n, seeds, row_ptr or mem_kind");
  if (first_step >= 0xfffffffeull) return fail(nullptr, CB_ERANGE, "first_step too large");
  int64_t N = 0, nrp = 0;
  for (int32_t i = 0; i < count; ++i) {
    if (n[i] < 0) return fail(nullptr, CB_EINVAL, "negative graph size");
    N += n[i] + (n[i] & 1);
    nrp += n[i] + 1;
  }
  if (N > 0x7fffffffLL) return fail(nullptr, CB_EINVAL, "batch exceeds 2^31-1 nodes");
  int rc;
  Graph* h = new_graph(cuda_stream, &rc);
  if (!h) return rc;
  auto bail = [&](int code) {
    g_error = h->last_error;
    destroy_graph(h);
    return code;
  };
  // every graph's offsets on the host: sizes and entry offsets
  const int64_t* rph = row_ptr;
  int64_t* rp_copy = nullptr;
  if (mem_kind == CB_DEVICE) {
    rp_copy = new (std::nothrow) int64_t[nrp];
    if (!rp_copy) return bail(fail(h, CB_ENOMEM, "host allocation failed"));
    if (cudaMemcpy(rp_copy, row_ptr, sizeof(int64_t) * nrp, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete[] rp_copy;
      return bail(fail(h, CB_EINVAL, "row_ptr is not readable device memory"));
    }
    rph = rp_copy;
  }
  h->nseg = count;
  h->hsegs = new (std::nothrow) Seg[count];
  int64_t* rpo = new (std::nothrow) int64_t[2 * static_cast<size_t>(count)];
  if (!h->hsegs || !rpo) {
    delete[] rp_copy;
    delete[] rpo;
    return bail(fail(h, CB_ENOMEM, "host allocation failed"));
  }
  int64_t* eoff = rpo + count;
  int64_t off = 0, r = 0, e = 0, base = 0, pairs = 0;
  bool bad = false;
  for (int32_t i = 0; i < count; ++i) {
    Seg& S = h->hsegs[i];
    S = Seg{};
    S.seed = seeds[i];
    S.off = off;
    S.n = n[i];
    S.span = n[i] + (n[i] & 1);
    S.bucket_base = base;
    S.B = bucket_bits(S.span);
    S.g = static_cast<uint32_t>(first_step);
    const int64_t z = rph[r + n[i]];
    bad |= rph[r] != 0 || z < 0 || (z & 1);
    for (int64_t l = 0; l < n[i] && !bad; ++l)   // offsets must not run backwards (they index col below)
      bad |= rph[r + l + 1] < rph[r + l];
    S.m = z / 2;
    S.pair_off = pairs;
    rpo[i] = r;
    eoff[i] = e;
    off += S.span;
    r += n[i] + 1;
    e += z;
    base += int64_t(1) << S.B;
    pairs += S.m;
  }
  delete[] rp_copy;
  if (bad || e / 2 >= (int64_t(1) << 32) || (e > 0 && !col)) {
    delete[] rpo;
    return bail(fail(h, CB_EINVAL, "each graph's row_ptr must start at 0, not decrease and end even"));
  }
  h->n = N;
  h->nnz = e;
  h->seed = seeds[0];
  h->g = first_step;
  h->nbuckets = base;
  h->inorder_threads = 256;   // many small graphs: many small deferred trades
  cudaStream_t s = h->stream;
  int64_t* d_rp_in = nullptr;
  int64_t* d_rpo = nullptr;
  if (dalloc(h, &h->segs, count) || dalloc(h, &h->seg_of, N) || dalloc(h, &h->rp_id, N + 1) || dalloc(h, &h->deg_id, N) ||
      dalloc(h, &h->col[0], e + kColPad) || dalloc(h, &h->col[1], e + kColPad) || dalloc(h, &h->err, 8) || dalloc(h, &h->counters, kCounters) ||
      !(h->host_counters = new (std::nothrow) int64_t[kCounters]) || dalloc(h, &d_rp_in, nrp) ||
      dalloc(h, &d_rpo, 2 * static_cast<int64_t>(count))) {
    delete[] rpo;
    dfree(h, d_rp_in);
    dfree(h, d_rpo);
    return bail(fail(h, CB_ENOMEM, "device allocation failed"));
  }
  const cudaMemcpyKind kind = mem_kind == CB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t ce = cudaMemsetAsync(h->err, 0, 8 * sizeof(int32_t), s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(h->segs, h->hsegs, sizeof(Seg) * count, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_rpo, rpo, sizeof(int64_t) * 2 * count, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_rp_in, row_ptr, sizeof(int64_t) * nrp, kind, s);
  if (ce == cudaSuccess && e) ce = cudaMemcpyAsync(h->col[0], col, sizeof(int32_t) * e, kind, s);
  if (ce == cudaSuccess && N) {
    k_fill_seg_of<<<grid1d(N, h->num_sms), 256, 0, s>>>(N, h->segs, count, h->seg_of);
    k_batch_offsets<<<grid1d(N + 1, h->num_sms), 256, 0, s>>>(N, h->segs, h->seg_of, d_rp_in, d_rpo, d_rpo + count,
                                                              e, h->rp_id, h->err);
    k_batch_cols<<<grid1d(N * 32, h->num_sms), 256, 0, s>>>(N, h->segs, h->seg_of, h->rp_id, h->col[0], h->err);
    h->launches += 3;
    ce = cudaGetLastError();
  } else if (ce == cudaSuccess) {
    ce = cudaMemsetAsync(h->rp_id, 0, sizeof(int64_t), s);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  delete[] rpo;
  dfree(h, d_rp_in);
  dfree(h, d_rpo);
  if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "batch import"));
  if ((rc = check_device_error(h))) {
    h->last_error = "a graph's row_ptr or ids are out of range";
    return bail(CB_EINVAL);
  }
  if ((rc = finish_create(h))) return bail(rc);
  *out = static_cast<cb_graph*>(h);
  return CB_OK;
}

int cb_global_trades(cb_handle h, uint32_t supersteps) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  if (h->g + supersteps >= 0xfffffffeull) return fail(h, CB_ERANGE, "super-step counter would pass 2^32-2");
  const int64_t launches0 = h->launches;
  // event sets still pending belong to the previous call
  for (int set = 0; set < 2; ++set) {
    const int rc = flush_timing(h, set, false);
    if (rc) return rc;
  }
  for (double& v : h->phase_ms) v = 0;
  if (h->use_graph && !h->timing && !h->swap_stats && !h->pres && supersteps > 0) {
    if (!h->step_exec[0]) {
      const int rc = capture_step_graphs(h);
      if (rc) return rc;
    }
    for (uint32_t i = 0; i < supersteps; ++i) {
      CB_CUDA(h, cudaGraphLaunch(h->step_exec[h->cur], h->stream));
      std::swap(h->col[0], h->col[1]);   // as super_step does
      h->cur = 1 - h->cur;
      h->g += 1;
      h->launches += h->step_launches;
    }
  } else {
    for (uint32_t i = 0; i < supersteps; ++i) {
      int rc = super_step(h);
      if (!rc && h->swap_stats) rc = count_swaps(h);
      if (!rc && h->pres) rc = record_presence(h);
      if (rc) return rc;
    }
  }
  h->stats[5] = h->launches - launches0;
  return CB_OK;
}

int cb_device_bytes(cb_handle h, int64_t* now, int64_t* peak) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  if (now) *now = h->dev_bytes;
  if (peak) *peak = h->dev_bytes_peak;
  return CB_OK;
}

int64_t cb_estimate_bytes(int64_t n, int64_t nnz, int64_t max_degree) {
  if (n < 0 || nnz < 0 || max_degree < 0) return fail(nullptr, CB_EINVAL, "negative size");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    sms = 152;
  return estimate_handle_bytes(n, nnz, max_degree, sms);
}

int cb_graph_count(cb_handle h) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  return h->nseg;
}

int cb_graph_info(cb_handle h, int32_t index, int64_t* n, int64_t* m) {
  if (!h || index < 0 || index >= h->nseg) return fail(h, CB_EINVAL, "bad handle or graph index");
  if (n) *n = h->hsegs[index].n;
  if (m) *m = h->hsegs[index].m;
  return CB_OK;
}

int cb_export_graph(cb_handle h, int32_t index, int32_t* edges, int64_t capacity_pairs, int64_t* m_out,
                    int mem_kind) {
  if (!h || !m_out || index < 0 || index >= h->nseg) return fail(h, CB_EINVAL, "bad handle, index or m_out");
  const Seg& S = h->hsegs[index];
  *m_out = S.m;
  if (!edges) return CB_OK;
  if (capacity_pairs < S.m) return fail(h, CB_ESIZE, "capacity below m");
  if (mem_kind != CB_HOST && mem_kind != CB_DEVICE) return fail(h, CB_EINVAL, "bad mem_kind");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  int rc;
  if ((rc = ensure_pairs(h))) return rc;
  return copy_pairs(h, S.pair_off, S.m, edges, mem_kind);
}

int cb_export_edges(cb_handle h, int32_t* edges, int64_t capacity_pairs, int64_t* m_out, int mem_kind) {
  if (!h || !m_out) return fail(h, CB_EINVAL, "NULL handle or m_out");
  *m_out = h->m;
  if (!edges) return CB_OK;
  if (capacity_pairs < h->m) return fail(h, CB_ESIZE, "capacity below m");
  if (mem_kind != CB_HOST && mem_kind != CB_DEVICE) return fail(h, CB_EINVAL, "bad mem_kind");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  int rc;
  if (h->nseg > 1) {   // every graph in turn, local ids
    if ((rc = ensure_pairs(h))) return rc;
    return copy_pairs(h, 0, h->m, edges, mem_kind);
  }
  int32_t* pairs = edges;
  if (mem_kind == CB_HOST) {
    CB_CUDA(h, dmalloc(h, reinterpret_cast<void**>(&pairs), sizeof(int32_t) * 2 * std::max<int64_t>(h->m, 1)));
  }
  rc = export_sorted_pairs(h, pairs);
  if (!rc && mem_kind == CB_HOST && h->m)
    rc = cudaMemcpyAsync(edges, pairs, sizeof(int32_t) * 2 * h->m, cudaMemcpyDeviceToHost, h->stream)
             ? fail(h, CB_ECUDA, "copy to host failed") : CB_OK;
  const int rc2 = check_device_error(h);
  if (mem_kind == CB_HOST) {
    dfree(h, pairs);
    h->dev_bytes -= static_cast<int64_t>(sizeof(int32_t) * 2 * std::max<int64_t>(h->m, 1));
  }
  return rc ? rc : rc2;
}

void cb_destroy(cb_handle h) {
  if (!h) return;
  release(h);
  delete h;
}

int cb_step(cb_handle h, uint64_t* g) {
  if (!h || !g) return fail(h, CB_EINVAL, "NULL argument");
  *g = h->g;
  return CB_OK;
}

int cb_sync(cb_handle h) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

const char* cb_last_error(cb_handle h) { return h ? h->last_error.c_str() : g_error.c_str(); }

int cb_info(cb_handle h, int64_t* n, int64_t* m) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  if (n) *n = h->n;
  if (m) *m = h->m;
  return CB_OK;
}

int cb_permutation(cb_handle h, uint64_t g, int32_t* order_out, int mem_kind) {
  if (!h || !order_out || (mem_kind != CB_HOST && mem_kind != CB_DEVICE)) return fail(h, CB_EINVAL, "bad argument");
  if (g >= 0xfffffffeull) return fail(h, CB_ERANGE, "step too large");
  int rc;
  // M is free between super steps
  if ((rc = compute_permutation(h, 0, static_cast<int64_t>(g), h->M, nullptr))) return rc;
  CB_CUDA(h, cudaMemcpyAsync(order_out, h->M, sizeof(int32_t) * h->n,
                             mem_kind == CB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
  return cb_sync(h);
}

int cb_stats(cb_handle h, int64_t* out, int count) {
  if (!h || !out || count < 0) return fail(h, CB_EINVAL, "bad argument");
  // counters of the last super step (reset at the start of each one)
  CB_CUDA(h, cudaMemcpyAsync(h->host_counters, h->counters, kCounters * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  const int64_t* hc = h->host_counters;
  // pass r + 1 runs what pass r left deferred (the last: the in-order pass)
  int64_t passes = 1;
  for (int r = 0; r <= h->retry_passes; ++r) passes += hc[kCtrPassLeft + r] > 0;
  h->stats[0] = passes;
  h->stats[1] = hc[kCtrPassLeft];
  h->stats[2] = h->stats[3] = 0;
  for (int k = 0; k < kClasses; ++k) h->stats[k < kWarpClasses ? 2 : 3] += hc[kCtrFirstLen + k];
  h->stats[4] = hc[kCtrGws];
  h->stats[6] = hc[kCtrPassLeft + h->retry_passes];
  for (int k = 0; k < kClasses; ++k) {
    h->stats[7 + k] = hc[kCtrFirstLen + k];
    h->stats[7 + kClasses + k] = hc[kCtrFirstEnt + k];
  }
  const int k = std::min(count, kStats);
  for (int i = 0; i < k; ++i) out[i] = h->stats[i];
  return k;
}

int cb_timings(cb_handle h, double* ms, int count) {
  if (!h || !ms || count < 0) return fail(h, CB_EINVAL, "bad argument");
  for (int set = 0; set < 2; ++set) {
    const int rc = flush_timing(h, set, true);
    if (rc) return rc;
  }
  const int k = std::min(count, kTimings);
  for (int i = 0; i < k; ++i) ms[i] = h->phase_ms[i];
  return k;
}

int cb_set_option(cb_handle h, const char* key, int64_t value) {
  if (!h || !key) return fail(h, CB_EINVAL, "bad argument");
  if (!std::strcmp(key, "cuda_graph")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "cuda_graph is 0 or 1");
    h->use_graph = value != 0;
    return CB_OK;
  }
  drop_step_graphs(h);   // every other option changes what a super step launches
  if (!std::strcmp(key, "tile_max")) {
    if (value < 0 || value > kTileMaxCap) return fail(h, CB_EINVAL, "tile_max out of range [0, 128]");
    h->tile_max = static_cast<int>(value);
    return size_trade_workspace(h);
  }
  if (!std::strcmp(key, "tile_paths")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "tile_paths is 0 or 1");
    h->tile_paths = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "presence")) {
    if (value < 0 || value > 1000000) return fail(h, CB_EINVAL, "presence out of range [0, 10^6]");
    return set_presence(h, value);
  }
  if (!std::strcmp(key, "wait_ms")) {
    if (value < 1 || value > 600000) return fail(h, CB_EINVAL, "wait_ms out of range [1, 600000]");
    h->wait_ns = h->uni_wait_ns = static_cast<uint64_t>(value) * 1000000ull;
    return CB_OK;
  }
  if (!std::strcmp(key, "hold_publish")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "hold_publish is 0 or 1");
    h->hold_publish = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "hold_trade")) {
    if (value < -1) return fail(h, CB_EINVAL, "hold_trade is -1 or a trade index");
    h->hold_trade = value;
    return CB_OK;
  }
  if (!std::strcmp(key, "fix_passes")) {
    if (value < 0 || value > 64) return fail(h, CB_EINVAL, "fix_passes out of range [0, 64]");
    h->fix_passes = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "cta_paths")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "cta_paths is 0 or 1");
    h->cta_paths = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "cand_max")) {
    if (value < 1 || value > 32) return fail(h, CB_EINVAL, "cand_max out of range [1, 32]");
    h->cand_max = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "block_max")) {
    if (value < 0 || value > kBlockMaxCap) return fail(h, CB_EINVAL, "block_max out of range [0, 2048]");
    h->block_max = static_cast<int>(value);
    return size_trade_workspace(h);
  }
  if (!std::strcmp(key, "smem_max")) {
    if (value < 64 || value > kSmemMaxCap) return fail(h, CB_EINVAL, "smem_max out of range [64, 8192]");
    h->smem_max = static_cast<int>(value);
    return size_trade_workspace(h);
  }
  if (!std::strcmp(key, "timing")) {
    if (value && !h->ev[0][0]) {
      for (auto& set : h->ev)
        for (auto& e : set) CB_CUDA(h, cudaEventCreate(&e));
    }
    h->timing = value != 0;
    return CB_OK;
  }
  if (!std::strcmp(key, "uniform_threads")) {
    if (value != 256 && value != 512 && value != 1024) return fail(h, CB_EINVAL, "uniform_threads is 256, 512 or 1024");
    h->uni_threads = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "lane_teams")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "lane_teams is 0 or 1");
    h->lane_teams = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "retry_passes")) {
    if (value < 0 || value > kRetryPassesMax) return fail(h, CB_EINVAL, "retry_passes out of range [0, 4]");
    h->retry_passes = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "inorder_threads")) {
    if (value != 256 && value != 1024) return fail(h, CB_EINVAL, "inorder_threads is 256 or 1024");
    h->inorder_threads = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "relaxed")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "relaxed is 0 or 1");
    return set_relaxed(h, value != 0);
  }
  if (!std::strcmp(key, "swap_stats")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "swap_stats is 0 or 1");
    return set_swap_stats(h, value != 0);
  }
  if (!std::strcmp(key, "wide_pack")) {
    if (value < 0 || value > 1) return fail(h, CB_EINVAL, "wide_pack is 0 or 1");
    h->wide_pack = value != 0;
    return CB_OK;
  }
  if (!std::strcmp(key, "bucket_cap")) {
    if (value < 2 || value > kBucketCapMax) return fail(h, CB_EINVAL, "bucket_cap out of range [2, 4096]");
    h->bucket_cap = static_cast<int>(value);
    return CB_OK;
  }
  return fail(h, CB_EINVAL, std::string("unknown option ") + key);
}

int cb_autotune(cb_handle h, uint32_t max_steps, int64_t* chosen, int count) {
  if (!h || count < 0) return fail(h, CB_EINVAL, "bad argument");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  if (h->g + max_steps >= 0xfffffffeull) return fail(h, CB_ERANGE, "super-step counter would pass 2^32-2");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CB_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, CB_ECUDA, "cudaEventCreate failed");
  }
  drop_step_graphs(h);
  const bool timing = h->timing;
  h->timing = false;
  uint32_t used = 0;
  int rc = CB_OK;
  // `per` super steps under the current options (fewer if the budget ends);
  // ms = their device time per step
  uint32_t per = 1;
  auto trial = [&](float* ms) -> int {
    if (cudaEventRecord(e0, h->stream) != cudaSuccess) return fail(h, CB_ECUDA, "cudaEventRecord failed");
    uint32_t k = 0;
    for (; k < per && used < max_steps; ++k, ++used) {
      const int r = super_step(h);
      if (r) return r;
    }
    if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return fail(h, CB_ECUDA, "event timing failed");
    *ms /= static_cast<float>(k ? k : 1);
    return CB_OK;
  };
  struct Knob {
    int* field;
    int cand[4];
    int ncand;
  };
  constexpr int kKnobs = 5;
  Knob knobs[kKnobs] = {{&h->tile_max, {32, 64, 128, 0}, 3},
                        {&h->block_max, {512, 1024, 2048, 0}, 3},
                        {&h->smem_max, {4096, 8192, 0, 0}, 2},
                        {&h->inorder_threads, {256, 1024, 0, 0}, 2},
                        {&h->retry_passes, {1, 2, 3, 0}, 3}};
  float ms = 0;
  if (used < max_steps) rc = trial(&ms);   // first launches load the kernels: not timed as a candidate
  {
    // the current settings, then every other candidate: super steps shared
    // evenly, at least one each
    int total = 1;
    for (const Knob& kn : knobs) total += kn.ncand;
    if (max_steps > used) per = std::max<uint32_t>(1, (max_steps - used) / static_cast<uint32_t>(total));
  }
  float best_ms = 3.4e38f;
  if (rc == CB_OK && used < max_steps) {
    rc = trial(&ms);
    if (rc == CB_OK) best_ms = ms;
  }
  // one knob at a time; a setting replaces the best one so far only when it
  // is at least 2 % faster (a step's time varies with its deferred trades)
  for (int k = 0; k < kKnobs && rc == CB_OK; ++k) {
    const int cur = *knobs[k].field;
    int best = cur;
    for (int j = 0; j < knobs[k].ncand && used < max_steps && rc == CB_OK; ++j) {
      if (knobs[k].cand[j] == cur) continue;
      *knobs[k].field = knobs[k].cand[j];
      rc = size_trade_workspace(h);   // the global workspace follows block_max and smem_max
      if (rc == CB_OK) rc = trial(&ms);
      if (rc == CB_OK && ms < 0.98f * best_ms) {
        best_ms = ms;
        best = knobs[k].cand[j];
      }
    }
    *knobs[k].field = best;
    if (rc == CB_OK) rc = size_trade_workspace(h);
  }
  h->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const int64_t vals[6] = {h->tile_max,        h->block_max, h->smem_max, h->inorder_threads,
                           static_cast<int64_t>(used), h->retry_passes};
  const int k = chosen ? std::min(count, 6) : 0;
  for (int i = 0; i < k; ++i) chosen[i] = vals[i];
  return k;
}

}  // extern "C"
