// Row-level utilities outside the super step: relabelling a CSR into another
// row order and node numbering (with each row sorted), input validation, the
// inverse of a permutation and the canonical edge export (Section 2: ordered
// edges [a,b], a<b).
#include <algorithm>

#include "cb_internal.cuh"
#include "team.cuh"

namespace cb {
namespace {

const int32_t kErrValidateHost = kErrValidate;

constexpr int kRowWarpMax = 256;     // rows up to this length: one warp
constexpr int kRowBlockSmem = 16384; // rows up to this length: one CTA in shared memory

__device__ __forceinline__ void latch(int32_t* err, int32_t code) { atomicCAS(err, 0, code); }

struct RowArgs {
  int64_t nrows;
  const int64_t* src_rp;
  const int32_t* src_col;
  const int32_t* rowmap;
  const int32_t* valmap;
  const int64_t* dst_rp;
  int32_t* dst_col;
  int32_t* err;
};

template <class Team>
__device__ void relabel_row(Team& tm, const RowArgs& a, int64_t q, int32_t* buf) {
  const int64_t x = a.rowmap ? a.rowmap[q] : q;
  const int64_t s0 = a.src_rp[x], len = a.src_rp[x + 1] - s0;
  const int64_t d0 = a.dst_rp[q];
  if (len != a.dst_rp[q + 1] - d0) {
    if (tm.rank == 0) latch(a.err, kErrRowLength);
    return;
  }
  const int P = next_pow2(static_cast<int>(len));
  for (int i = tm.rank; i < P; i += Team::N) {
    int32_t v = 0x7fffffff;
    if (i < len) {
      v = a.src_col[s0 + i];
      if (a.valmap) v = a.valmap[v];
    }
    buf[i] = v;
  }
  tm.sync();
  team_bitonic_sort(tm, buf, P);
  for (int i = tm.rank; i < len; i += Team::N) a.dst_col[d0 + i] = buf[i];
  tm.sync();
}

__global__ void __launch_bounds__(256) k_rows_warp(RowArgs a) {
  __shared__ int32_t buf[8][kRowWarpMax];
  WarpTeam tm;
  const int w = threadIdx.x >> 5;
  const int64_t nw = int64_t(gridDim.x) * 8;
  for (int64_t q = blockIdx.x * int64_t(8) + w; q < a.nrows; q += nw) {
    const int64_t len = a.dst_rp[q + 1] - a.dst_rp[q];
    if (len > kRowWarpMax) continue;
    relabel_row(tm, a, q, buf[w]);
  }
}

// Long rows: one CTA per row, shared memory or a global slice per CTA.
__global__ void __launch_bounds__(256) k_rows_block(RowArgs a, int32_t* gws, int64_t slice) {
  extern __shared__ int32_t sbuf[];
  __shared__ int64_t red[BlockTeam<256>::kRedSlots];
  BlockTeam<256> tm(red);
  for (int64_t q = blockIdx.x; q < a.nrows; q += gridDim.x) {
    const int64_t len = a.dst_rp[q + 1] - a.dst_rp[q];
    if (len <= kRowWarpMax) continue;
    int32_t* buf = (len <= kRowBlockSmem) ? sbuf : gws + slice * blockIdx.x;
    relabel_row(tm, a, q, buf);
  }
}

__global__ void k_check_rp(int64_t n, const int64_t* __restrict__ rp, int32_t* err) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t d = rp[x + 1] - rp[x];
    if (d < 0 || d >= n || (x == 0 && rp[0] != 0)) latch(err, kErrValidate);
  }
}

// Rows sorted: strictly increasing, in range, no self loop, and symmetric.
// Symmetry with half the searches: every entry y > x must find x in row y;
// those mirrors are distinct entries below the diagonal, so the graph is
// symmetric exactly when, in addition, there are as many entries below the
// diagonal as above (counted into ud[0] and ud[1]).
__global__ void k_validate(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           int32_t* err, unsigned long long* ud) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  unsigned long long up = 0, down = 0;
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < n; x += nw) {
    const int64_t b = rp[x], e = rp[x + 1];
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t y = col[i];
      bool bad = y < 0 || y >= n || y == x || (i > b && col[i - 1] >= y);
      if (!bad && y > x) {
        ++up;
        const int64_t yb = rp[y], ye = rp[y + 1];
        const int k = lower_bound(col + yb, static_cast<int>(ye - yb), static_cast<int32_t>(x));
        bad = (yb + k >= ye) || col[yb + k] != x;
      } else if (!bad) {
        ++down;
      }
      if (bad) latch(err, kErrValidate);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    up += __shfl_xor_sync(kFull, up, o);
    down += __shfl_xor_sync(kFull, down, o);
  }
  if (lane == 0) {
    if (up) atomicAdd(&ud[0], up);
    if (down) atomicAdd(&ud[1], down);
  }
}

// err <- kErrValidate unless every row is strictly increasing (sorted input).
__global__ void k_rows_sorted(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* flag) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  bool unsorted = false;
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < n; x += nw) {
    const int64_t b = rp[x], e = rp[x + 1];
    for (int64_t i = b + 1 + lane; i < e; i += 32) unsorted |= col[i - 1] >= col[i];
  }
  if (__any_sync(kFull, unsorted) && lane == 0) atomicExch(flag, 1);
}

// dst row q <- src row rowmap[q], values mapped through valmap, order kept.
__global__ void k_relabel(RowArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; q < a.nrows; q += nw) {
    const int64_t x = a.rowmap ? a.rowmap[q] : q;
    const int64_t s0 = a.src_rp[x], len = a.src_rp[x + 1] - s0;
    const int64_t d0 = a.dst_rp[q];
    if (len != a.dst_rp[q + 1] - d0) {
      if (lane == 0) latch(a.err, kErrRowLength);
      continue;
    }
    for (int64_t i = lane; i < len; i += 32) {
      const int32_t v = a.src_col[s0 + i];
      a.dst_col[d0 + i] = a.valmap ? a.valmap[v] : v;
    }
  }
}

__global__ void k_invert(int64_t n, const int32_t* __restrict__ order, int32_t* __restrict__ pos) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x)
    pos[order[p]] = static_cast<int32_t>(p);
}

// entries of row x greater than x (rows sorted ascending)
__global__ void k_count_upper(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* __restrict__ cnt) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = rp[x], len = rp[x + 1] - b;
    const int k = lower_bound(col + b, static_cast<int>(len), static_cast<int32_t>(x + 1));
    cnt[x] = static_cast<int32_t>(len - k);
  }
}

// Pairs (x, y) with x < y, ids local to x's graph (both ends share it).
__global__ void k_write_pairs(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ cnt, const int64_t* __restrict__ off,
                              const Seg* __restrict__ segs, const int32_t* __restrict__ seg_of,
                              int32_t* __restrict__ pairs) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < n; x += nw) {
    const int64_t e = rp[x + 1], c = cnt[x], b = e - c, o = off[x];
    const int32_t base = seg_of ? static_cast<int32_t>(segs[seg_of[x]].off) : 0;
    for (int64_t i = lane; i < c; i += 32) {
      pairs[2 * (o + i)] = static_cast<int32_t>(x) - base;
      pairs[2 * (o + i) + 1] = col[b + i] - base;
    }
  }
}

unsigned grid_of(int64_t work, int threads, int num_sms) {
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = int64_t(num_sms) * 16;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min(want, cap)));
}

}  // namespace

int permute_rows(Graph* h, int64_t nrows, const int64_t* src_rp, const int32_t* src_col,
                 const int32_t* rowmap, const int32_t* valmap, const int64_t* dst_rp, int32_t* dst_col) {
  if (nrows == 0) return CB_OK;
  RowArgs a{nrows, src_rp, src_col, rowmap, valmap, dst_rp, dst_col, h->err};
  const unsigned wgrid = grid_of(nrows, 8, h->num_sms);
  k_rows_warp<<<wgrid, 256, 0, h->stream>>>(a);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  if (h->maxdeg > kRowWarpMax) {
    // global slice per CTA for rows longer than the shared-memory buffer
    int64_t slice = 0;
    int ctas = h->num_sms * 2;
    int32_t* gws = nullptr;
    if (h->maxdeg > kRowBlockSmem) {
      slice = next_pow2_host(h->maxdeg);
      const size_t budget = h->ws_slice * static_cast<size_t>(h->ws_ctas);
      ctas = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ctas, budget / (slice * 4))));
      if (budget < static_cast<size_t>(slice) * 4) return fail(h, CB_ENOMEM, "row workspace too small");
      gws = static_cast<int32_t*>(h->ws_global);
    }
    CB_CUDA(h, cudaFuncSetAttribute(k_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kRowBlockSmem * 4));
    k_rows_block<<<ctas, 256, kRowBlockSmem * 4, h->stream>>>(a, gws, slice);
    CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  }
  return CB_OK;
}

int validate_sorted_graph(Graph* h, const int64_t* rp, const int32_t* col, int64_t n) {
  if (n == 0) return CB_OK;
  unsigned long long* ud = reinterpret_cast<unsigned long long*>(h->counters) + 6;
  CB_CUDA(h, cudaMemsetAsync(ud, 0, 2 * sizeof(unsigned long long), h->stream));
  k_validate<<<grid_of(n * 32, 256, h->num_sms), 256, 0, h->stream>>>(n, rp, col, h->err, ud);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  unsigned long long hud[2] = {0, 0};
  CB_CUDA(h, cudaMemcpyAsync(hud, ud, sizeof(hud), cudaMemcpyDeviceToHost, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (hud[0] != hud[1]) {
    CB_CUDA(h, cudaMemcpyAsync(h->err, &kErrValidateHost, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  }
  return CB_OK;
}

int rows_sorted(Graph* h, const int64_t* rp, const int32_t* col, int64_t n, bool* sorted) {
  *sorted = true;
  if (n == 0) return CB_OK;
  int32_t* flag = reinterpret_cast<int32_t*>(h->counters + 8);
  CB_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(int32_t), h->stream));
  k_rows_sorted<<<grid_of(n * 32, 256, h->num_sms), 256, 0, h->stream>>>(n, rp, col, flag);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  int32_t hf = 0;
  CB_CUDA(h, cudaMemcpyAsync(&hf, flag, sizeof(hf), cudaMemcpyDeviceToHost, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  *sorted = hf == 0;
  return CB_OK;
}

int relabel_rows(Graph* h, int64_t nrows, const int64_t* src_rp, const int32_t* src_col, const int32_t* rowmap,
                 const int32_t* valmap, const int64_t* dst_rp, int32_t* dst_col) {
  if (nrows == 0) return CB_OK;
  RowArgs a{nrows, src_rp, src_col, rowmap, valmap, dst_rp, dst_col, h->err};
  k_relabel<<<grid_of(nrows * 32, 256, h->num_sms), 256, 0, h->stream>>>(a);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

int check_row_offsets(Graph* h, const int64_t* rp, int64_t n) {
  if (n == 0) return CB_OK;
  k_check_rp<<<grid_of(n, 256, h->num_sms), 256, 0, h->stream>>>(n, rp, h->err);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

int invert_permutation(Graph* h, const int32_t* order, int32_t* pos) {
  if (h->n == 0) return CB_OK;
  k_invert<<<grid_of(h->n, 256, h->num_sms), 256, 0, h->stream>>>(h->n, order, pos);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

int export_pairs(Graph* h, const int64_t* rp, const int32_t* col, int32_t* pairs) {
  const int64_t n = h->n;
  if (n == 0) return CB_OK;
  int32_t* cnt = h->deg_next;      // free between super steps
  int64_t* off = h->rp[1 - h->cur];
  k_count_upper<<<grid_of(n, 256, h->num_sms), 256, 0, h->stream>>>(n, rp, col, cnt);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(cnt, off, n, h->scan_ws, h->stream, &h->launches));
  k_write_pairs<<<grid_of(n * 32, 256, h->num_sms), 256, 0, h->stream>>>(n, rp, col, cnt, off, h->segs, h->seg_of,
                                                                           pairs);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

}  // namespace cb
