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

template <class T>
cudaError_t dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * static_cast<size_t>(count));
}

void release(Graph* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  void* bufs[] = {h->deg_id, h->rp_id, h->order[0], h->order[1], h->rp[0], h->rp[1], h->col[0], h->col[1],
                  h->pos_next, h->M, h->deg_next, h->stash, h->thr_key, h->thr_tb, h->thr_top, h->done,
                  h->list[0], h->list[1], h->list[2], h->tile_off, h->tile_first, h->cls_flag, h->cls_scan,
                  h->list_def[0], h->list_def[1], h->counters, h->err,
                  h->ws_global, h->sort_ws, h->scan_ws};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h->host_counters) cudaFreeHost(h->host_counters);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Read the latched device error word; synchronises the stream.
int check_device_error(Graph* h) {
  int32_t e = 0;
  CB_CUDA(h, cudaMemcpyAsync(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (e != kErrNone) {
    h->latched = CB_ECHECK;
    return fail(h, CB_ECHECK, "device check failed (code " + std::to_string(e) + ")");
  }
  return CB_OK;
}

int size_trade_workspace(Graph* h) {
  if (h->ws_global) {
    cudaFree(h->ws_global);
    h->ws_global = nullptr;
  }
  const int64_t max_trade = 2 * h->maxdeg;
  h->ws_ctas = h->num_sms * 4;
  h->ws_slice = 0;
  if (max_trade > h->smem_max || h->maxdeg > 16384) {
    h->ws_slice = trade_ws_slice_bytes(std::max<int64_t>(max_trade, 1));
    const size_t budget = size_t(2) << 30;
    h->ws_ctas = static_cast<int>(std::max<size_t>(1, std::min<size_t>(h->num_sms * 2, budget / h->ws_slice)));
    CB_CUDA(h, cudaMalloc(&h->ws_global, h->ws_slice * h->ws_ctas));
  }
  return CB_OK;
}

}  // namespace

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

using namespace cb;

extern "C" {

int cb_create(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed, uint64_t first_step,
              int mem_kind, void* cuda_stream, cb_handle* out) {
  if (!out) return fail(nullptr, CB_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0 || n > 0x7fffffffLL || !row_ptr || (mem_kind != CB_HOST && mem_kind != CB_DEVICE))
    return fail(nullptr, CB_EINVAL, "bad n, row_ptr or mem_kind");
  if (first_step >= 0xfffffffeull) return fail(nullptr, CB_ERANGE, "first_step too large");
  cb_graph* h = new (std::nothrow) cb_graph();
  if (!h) return fail(nullptr, CB_ENOMEM, "host allocation failed");
  auto bail = [&](int rc) {
    g_error = h->last_error;
    release(h);
    delete h;
    return rc;
  };
  CB_CUDA(h, cudaGetDevice(&h->device)) ;
  CB_CUDA(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(h, CB_ECUDA, "stream creation failed"));
    h->own_stream = true;
  }
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
  h->m = nnz / 2;
  h->T = n / 2;
  h->ntasks = h->T + (n & 1);
  h->seed = seed;
  h->g = first_step;
  cudaStream_t s = h->stream;
  int rc;
  if (dalloc(&h->rp_id, n + 1) || dalloc(&h->deg_id, n) || dalloc(&h->col[0], nnz) || dalloc(&h->col[1], nnz) ||
      dalloc(&h->err, 8) || dalloc(&h->counters, kCounters) ||
      cudaMallocHost(&h->host_counters, kCounters * sizeof(int64_t)))
    return bail(fail(h, CB_ENOMEM, "device allocation failed"));
  CB_CUDA(h, cudaMemsetAsync(h->err, 0, 8 * sizeof(int32_t), s));
  CB_CUDA(h, cudaMemcpyAsync(h->rp_id, row_ptr, sizeof(int64_t) * (n + 1), kind, s));
  if (nnz) CB_CUDA(h, cudaMemcpyAsync(h->col[0], col, sizeof(int32_t) * nnz, kind, s));
  if ((rc = check_row_offsets(h, h->rp_id, n))) return bail(rc);
  {
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(h->counters);
    CB_CUDA(h, cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
    if (n) k_degrees<<<grid1d(n, h->num_sms), 256, 0, s>>>(n, h->rp_id, h->deg_id, dmax);
    CB_CUDA(h, cudaGetLastError());
  ++h->launches;
    unsigned long long hm = 0;
    CB_CUDA(h, cudaMemcpyAsync(&hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, s));
    if ((rc = check_device_error(h))) {
      h->last_error = "row_ptr is not a valid CSR offset array (degrees must be in [0, n))";
      return bail(CB_EINVAL);
    }
    h->maxdeg = static_cast<int64_t>(hm);
  }
  h->sort_ws_bytes = perm_ws_bytes(std::max<int64_t>(n, 1));
  h->scan_ws_bytes = scan_ws_bytes(n + 1);
  int64_t def_cap = 1;   // the in-order resolver bitonic-sorts a deferred list padded to a power of two
  while (def_cap < h->ntasks) def_cap <<= 1;
  if (dalloc(&h->order[0], n) || dalloc(&h->order[1], n) || dalloc(&h->rp[0], n + 1) || dalloc(&h->rp[1], n + 1) ||
      dalloc(&h->pos_next, n) || dalloc(&h->M, n) || dalloc(&h->deg_next, n) || dalloc(&h->stash, nnz) ||
      dalloc(&h->thr_key, h->ntasks) || dalloc(&h->thr_tb, h->ntasks) || dalloc(&h->done, h->ntasks) ||
      dalloc(&h->thr_top, h->ntasks) || dalloc(&h->list[0], h->ntasks) || dalloc(&h->list[1], h->ntasks) ||
      dalloc(&h->list[2], h->ntasks) || dalloc(&h->tile_off, h->ntasks) || dalloc(&h->tile_first, h->ntasks + 2) || dalloc(&h->cls_flag, 4 * h->ntasks) ||
      dalloc(&h->cls_scan, 4 * (h->ntasks + 1)) || dalloc(&h->list_def[0], def_cap) ||
      dalloc(&h->list_def[1], def_cap) ||
      cudaMalloc(&h->sort_ws, h->sort_ws_bytes) || cudaMalloc(&h->scan_ws, h->scan_ws_bytes))
    return bail(fail(h, CB_ENOMEM, "device allocation failed"));
  CB_CUDA(h, cudaMemsetAsync(h->done, 0, sizeof(uint32_t) * std::max<int64_t>(h->ntasks, 1), s));
  if ((rc = size_trade_workspace(h))) return bail(rc);
  // sort every row (id space) into col[1] and validate: simple and symmetric
  if ((rc = permute_rows(h, n, h->rp_id, h->col[0], nullptr, nullptr, h->rp_id, h->col[1]))) return bail(rc);
  if ((rc = validate_sorted_graph(h, h->rp_id, h->col[1], n))) return bail(rc);
  if ((rc = check_device_error(h))) {
    h->last_error = "graph is not simple and symmetric";
    return bail(CB_EINVAL);
  }
  // position-space layout of the first super step
  h->cur = 0;
  if ((rc = compute_permutation(h, h->g, h->order[0], h->pos_next))) return bail(rc);
  if (n) k_gather_deg<<<grid1d(n, h->num_sms), 256, 0, s>>>(n, h->order[0], h->deg_id, h->deg_next);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(h->deg_next, h->rp[0], n, h->scan_ws, s, &h->launches));
  if ((rc = permute_rows(h, n, h->rp_id, h->col[1], h->order[0], h->pos_next, h->rp[0], h->col[0]))) return bail(rc);
  if ((rc = check_device_error(h))) return bail(rc);
  *out = h;
  return CB_OK;
}

int cb_global_trades(cb_handle h, uint32_t supersteps) {
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  if (h->g + supersteps >= 0xfffffffeull) return fail(h, CB_ERANGE, "super-step counter would pass 2^32-2");
  const int64_t launches0 = h->launches;
  for (double& v : h->phase_ms) v = 0;
  for (uint32_t i = 0; i < supersteps; ++i) {
    const int rc = super_step(h);
    if (rc) return rc;
  }
  h->stats[5] = h->launches - launches0;
  return CB_OK;
}

int cb_export_edges(cb_handle h, int32_t* edges, int64_t capacity_pairs, int64_t* m_out, int mem_kind) {
  if (!h || !m_out) return fail(h, CB_EINVAL, "NULL handle or m_out");
  *m_out = h->m;
  if (!edges) return CB_OK;
  if (capacity_pairs < h->m) return fail(h, CB_ESIZE, "capacity below m");
  if (mem_kind != CB_HOST && mem_kind != CB_DEVICE) return fail(h, CB_EINVAL, "bad mem_kind");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  int rc;
  const int spare = 1 - h->cur;
  if ((rc = invert_permutation(h, h->order[h->cur], h->pos_next))) return rc;
  if ((rc = permute_rows(h, h->n, h->rp[h->cur], h->col[h->cur], h->pos_next, h->order[h->cur], h->rp_id,
                         h->col[spare])))
    return rc;
  int32_t* pairs = edges;
  if (mem_kind == CB_HOST) {
    CB_CUDA(h, cudaMalloc(&pairs, sizeof(int32_t) * 2 * std::max<int64_t>(h->m, 1)));
  }
  rc = export_pairs(h, h->rp_id, h->col[spare], pairs);
  if (!rc && mem_kind == CB_HOST && h->m)
    rc = cudaMemcpyAsync(edges, pairs, sizeof(int32_t) * 2 * h->m, cudaMemcpyDeviceToHost, h->stream)
             ? fail(h, CB_ECUDA, "copy to host failed") : CB_OK;
  const int rc2 = check_device_error(h);
  if (mem_kind == CB_HOST) cudaFree(pairs);
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
  if ((rc = compute_permutation(h, g, h->M, nullptr))) return rc;
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
  int64_t passes = 1, deferred = 0;
  for (int i = 1; i < kPassSlots && i < h->last_passes_queued; ++i) {
    if (hc[8 + i] == 0) break;
    deferred += hc[8 + i];
    passes = i + 1;
  }
  const int64_t left = hc[4 + h->last_in];   // run by the resolver
  if (left) {
    deferred += left;
    passes += 1;
  }
  h->stats[0] = passes;
  h->stats[1] = deferred;
  h->stats[2] = hc[0];
  h->stats[3] = hc[1] + hc[2];
  h->stats[4] = hc[kCounters - 1];
  const int k = std::min(count, 6);
  for (int i = 0; i < k; ++i) out[i] = h->stats[i];
  return k;
}

int cb_timings(cb_handle h, double* ms, int count) {
  if (!h || !ms || count < 0) return fail(h, CB_EINVAL, "bad argument");
  const int k = std::min(count, 4);
  for (int i = 0; i < k; ++i) ms[i] = h->phase_ms[i];
  return k;
}

int cb_set_option(cb_handle h, const char* key, int64_t value) {
  if (!h || !key) return fail(h, CB_EINVAL, "bad argument");
  if (!std::strcmp(key, "tile_max")) {
    if (value < 0 || value > kTileMaxCap) return fail(h, CB_EINVAL, "tile_max out of range [0, 128]");
    h->tile_max = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "queued_passes")) {
    if (value < 0 || value > 64) return fail(h, CB_EINVAL, "queued_passes out of range [0, 64]");
    h->queued_passes = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "tile_paths")) {
    if (value < 0 || value > 3) return fail(h, CB_EINVAL, "tile_paths out of range [0, 3]");
    h->tile_paths = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "block_max")) {
    if (value < 0 || value > kBlockMaxCap) return fail(h, CB_EINVAL, "block_max out of range [0, 2048]");
    h->block_max = static_cast<int>(value);
    return CB_OK;
  }
  if (!std::strcmp(key, "smem_max")) {
    if (value < 64 || value > kSmemMaxCap) return fail(h, CB_EINVAL, "smem_max out of range [64, 8192]");
    h->smem_max = static_cast<int>(value);
    return size_trade_workspace(h);
  }
  if (!std::strcmp(key, "timing")) {
    if (value && !h->ev[0]) {
      for (auto& e : h->ev) CB_CUDA(h, cudaEventCreate(&e));
    }
    h->timing = value != 0;
    return CB_OK;
  }
  if (!std::strcmp(key, "bucket_cap")) {
    if (value < 2 || value > 4096) return fail(h, CB_EINVAL, "bucket_cap out of range [2, 4096]");
    h->bucket_cap = static_cast<int>(value);
    return CB_OK;
  }
  return fail(h, CB_EINVAL, std::string("unknown option ") + key);
}

}  // extern "C"
