// Row-level utilities outside the super step: relabelling a CSR into another
// row order and node numbering (with each row sorted), input validation, the
// inverse of a permutation and the canonical edge export (Section 2: ordered
// edges [a,b], a<b).
#include <algorithm>

#include "cb_internal.cuh"
#include "team.cuh"

namespace cb {
namespace {

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

// Validation of sorted rows: strictly increasing, in range, no self loop,
// and symmetric.  Symmetry is checked exactly:
//   - every entry y > x of row x must be found among the entries of row y
//     below the diagonal (L_y);
//   - the entries above the diagonal, summed over all rows, must be as many
//     as those below.
// The found entries are distinct (rows are strictly increasing), so each L_y
// holds at least as many as point into it, and the totals force equality.
// For locality the upper entries are first partitioned into buckets of
// target rows, with one reservation per bucket and CTA. Each bucket's
// searches then stay within a few MB of rows that L2 holds.

constexpr int kVBuckets = 4096;     // target-row buckets of the partition

// Entry i of row x (rows [b, e)): its id if it lies above the diagonal and
// the row is well formed up to it, -1 otherwise; *bad for a malformed entry.
// Every pass of the partition uses this one predicate, so counts, space and
// writes agree on any input.
__device__ __forceinline__ int32_t upper_entry(const int32_t* __restrict__ col, int64_t b, int64_t i, int64_t x,
                                               int64_t n, bool* bad) {
  const int32_t y = col[i];
  *bad = y < 0 || y >= n || y == x || (i > b && col[i - 1] >= y);
  return (!*bad && y > x) ? y : -1;
}

// low[x] = entries of row x below x (a lower bound in the sorted row)
__global__ void k_lower_count(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* __restrict__ low) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x)
    low[x] = lower_bound(col + rp[x], static_cast<int>(rp[x + 1] - rp[x]), static_cast<int32_t>(x));
}

// Row checks and the partition: each CTA takes a contiguous range of rows,
// counts its upper entries per bucket, reserves their space with one atomic
// per bucket, and writes (x, y) into it.
__global__ void __launch_bounds__(256) k_vpart(int64_t n, const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ col, int sh,
                                               unsigned long long* __restrict__ cursor, int2* __restrict__ part,
                                               unsigned long long cap, int32_t* err) {
  __shared__ int32_t cnt[kVBuckets];
  __shared__ unsigned long long base[kVBuckets];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
  for (int b = threadIdx.x; b < kVBuckets; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  for (int64_t x = r0 + w; x < r1; x += blockDim.x >> 5) {
    const int64_t b = rp[x], e = rp[x + 1];
    for (int64_t i = b + lane; i < e; i += 32) {
      bool bad;
      const int32_t y = upper_entry(col, b, i, x, n, &bad);
      if (bad) latch(err, kErrValidate);
      else if (y >= 0) atomicAdd(&cnt[y >> sh], 1);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kVBuckets; b += blockDim.x) {
    base[b] = cnt[b] ? atomicAdd(&cursor[b], static_cast<unsigned long long>(cnt[b])) : 0;
    cnt[b] = 0;
  }
  __syncthreads();
  for (int64_t x = r0 + w; x < r1; x += blockDim.x >> 5) {
    const int64_t b = rp[x], e = rp[x + 1];
    for (int64_t i = b + lane; i < e; i += 32) {
      bool bad;
      const int32_t y = upper_entry(col, b, i, x, n, &bad);
      if (y >= 0) {
        const int k = y >> sh;
        const unsigned long long slot = base[k] + static_cast<unsigned long long>(atomicAdd(&cnt[k], 1));
        if (slot < cap) part[slot] = make_int2(static_cast<int32_t>(x), y);
        else latch(err, kErrValidate);   // more entries above the diagonal than a symmetric graph has
      }
    }
  }
}

// Every partitioned (x, y) found in L_y; and as many entries above the
// diagonal as below (bucket space boff[nb] against the scan of low, grp[n]).
// A thread runs kSearchLanes binary searches in lockstep, so that many loads
// are in flight per step: a single search is a chain of dependent L2 reads.
constexpr int kSearchLanes = 8;

__global__ void k_vcheck(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const int32_t* __restrict__ low, const int2* __restrict__ part,
                         const int64_t* __restrict__ boff, int nb, const int64_t* __restrict__ grp, int64_t cap,
                         int32_t* err) {
  const int64_t all = boff[nb];
  if (blockIdx.x == 0 && threadIdx.x == 0 && all != grp[n]) latch(err, kErrValidate);
  const int64_t total = all < cap ? all : cap;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x * kSearchLanes;
  for (int64_t i0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) * kSearchLanes; i0 < total; i0 += stride) {
    const int32_t* row[kSearchLanes];
    int32_t key[kSearchLanes];
    int lo[kSearchLanes], hi[kSearchLanes], ly[kSearchLanes];
#pragma unroll
    for (int j = 0; j < kSearchLanes; ++j) {
      lo[j] = 0;
      hi[j] = 0;
      ly[j] = 0;
      key[j] = 0;
      row[j] = col;
      if (i0 + j >= total) continue;
      const int2 p = part[i0 + j];
      if (p.x < 0 || p.y <= p.x || p.y >= n) {   // a slot no valid entry wrote (malformed input)
        latch(err, kErrValidate);
        continue;
      }
      row[j] = col + rp[p.y];
      key[j] = p.x;
      ly[j] = low[p.y];
      hi[j] = ly[j];
      lo[j] = 0;
      if (ly[j] == 0) latch(err, kErrValidate);   // nothing below the diagonal to find x in
    }
    for (;;) {
      bool more = false;
#pragma unroll
      for (int j = 0; j < kSearchLanes; ++j) {
        if (lo[j] < hi[j]) {
          more = true;
          const int mid = (lo[j] + hi[j]) >> 1;
          if (row[j][mid] < key[j]) lo[j] = mid + 1;
          else hi[j] = mid;
        }
      }
      if (!more) break;
    }
#pragma unroll
    for (int j = 0; j < kSearchLanes; ++j)
      if (ly[j] > 0 && (lo[j] >= ly[j] || row[j][lo[j]] != key[j])) latch(err, kErrValidate);
  }
}

// bucket offsets from the scanned counts; the cursor starts at each offset
__global__ void k_vcursor(int nb, const int64_t* __restrict__ boff, unsigned long long* __restrict__ cursor) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
    cursor[b] = static_cast<unsigned long long>(boff[b]);
}

// upper entries per bucket (row checks come with the partition)
__global__ void __launch_bounds__(256) k_vcount(int64_t n, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, int sh, int32_t* __restrict__ hist) {
  __shared__ int32_t cnt[kVBuckets];
  for (int b = threadIdx.x; b < kVBuckets; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < n; x += nw)
    for (int64_t i = rp[x] + lane; i < rp[x + 1]; i += 32) {
      bool bad;
      const int32_t y = upper_entry(col, rp[x], i, x, n, &bad);
      if (y >= 0) atomicAdd(&cnt[y >> sh], 1);
    }
  __syncthreads();
  for (int b = threadIdx.x; b < kVBuckets; b += blockDim.x)
    if (cnt[b]) atomicAdd(&hist[b], cnt[b]);
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

// ---- canonical export: only the entries above the diagonal are sorted

// cnt[x] = entries of (unsorted) row x greater than x
__global__ void k_count_above(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t x = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; x < n; x += nw) {
    int c = 0;
    for (int64_t i = rp[x] + lane; i < rp[x + 1]; i += 32) c += col[i] > x;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) cnt[x] = c;
  }
}

struct AboveArgs {
  int64_t n;
  const int64_t* rp;
  const int32_t* col;
  const int32_t* cnt;
  const int64_t* off;
  const Seg* segs;
  const int32_t* seg_of;
  int32_t* pairs;
  int32_t* err;
};

// Row x's entries above x, compacted into buf, sorted, written as pairs
// (x, y) with ids local to x's graph.
template <class Team>
__device__ void sort_above(Team& tm, const AboveArgs& a, int64_t x, int32_t* buf) {
  const int64_t b = a.rp[x], len = a.rp[x + 1] - b;
  const int c = a.cnt[x];
  const int P = next_pow2(c > 1 ? c : 1);
  int64_t base = 0;
  for (int64_t r0 = 0; r0 < len; r0 += Team::N) {
    const int64_t i = r0 + tm.rank;
    const int32_t v = i < len ? a.col[b + i] : -1;
    const bool up = v > x;
    const int64_t pos = tm.exscan(up ? 1 : 0);
    if (up && base + pos < c) buf[base + pos] = v;
    base += tm.sum(up ? 1 : 0);
  }
  if (base != c && tm.rank == 0) latch(a.err, kErrRowLength);
  for (int i = c + tm.rank; i < P; i += Team::N) buf[i] = 0x7fffffff;
  tm.sync();
  team_bitonic_sort(tm, buf, P);
  const int32_t sb = a.seg_of ? static_cast<int32_t>(a.segs[a.seg_of[x]].off) : 0;
  const int64_t o = a.off[x];
  for (int i = tm.rank; i < c; i += Team::N) {
    a.pairs[2 * (o + i)] = static_cast<int32_t>(x) - sb;
    a.pairs[2 * (o + i) + 1] = buf[i] - sb;
  }
  tm.sync();
}

// rows with at most kRowWarpMax entries above the diagonal: one warp each
__global__ void __launch_bounds__(256) k_above_warp(AboveArgs a) {
  __shared__ int32_t buf[8][kRowWarpMax];
  WarpTeam tm;
  const int w = threadIdx.x >> 5;
  const int64_t nw = int64_t(gridDim.x) * 8;
  for (int64_t x = blockIdx.x * int64_t(8) + w; x < a.n; x += nw)
    if (a.cnt[x] <= kRowWarpMax) sort_above(tm, a, x, buf[w]);
}

// rows with lo < entries above the diagonal <= hi: one CTA each, in `cap`
// ints of shared memory or, above that, a global slice per CTA
__global__ void __launch_bounds__(256) k_above_block(AboveArgs a, int lo, int64_t hi, int cap, int32_t* gws,
                                                     int64_t slice) {
  extern __shared__ int32_t sbuf[];
  __shared__ int64_t red[BlockTeam<256>::kRedSlots];
  BlockTeam<256> tm(red);
  for (int64_t x = blockIdx.x; x < a.n; x += gridDim.x) {
    const int c = a.cnt[x];
    if (c <= lo || c > hi) continue;
    sort_above(tm, a, x, c <= cap ? sbuf : gws + slice * blockIdx.x);
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

int validate_sorted_graph(Graph* h, const int64_t* rp, const int32_t* col, int64_t n, int32_t* grouped) {
  if (n == 0) return CB_OK;
  cudaStream_t s = h->stream;
  // scratch: low in a step buffer of n int32, its scan in rp[1] (n+1 int64),
  // none in use before the first super step; the partition in `grouped`
  int32_t* low = h->M;
  int64_t* grp = h->rp[1];
  int sh = 0;
  while (((n - 1) >> sh) >= kVBuckets) ++sh;
  const int nb = static_cast<int>(((n - 1) >> sh) + 1);
  char* ws = nullptr;
  const size_t ws_bytes = sizeof(int32_t) * kVBuckets + sizeof(int64_t) * (kVBuckets + 1) +
                          sizeof(unsigned long long) * kVBuckets + scan_ws_bytes(kVBuckets) + 64;
  CB_CUDA(h, dev_alloc(h, reinterpret_cast<void**>(&ws), ws_bytes));
  int32_t* hist = reinterpret_cast<int32_t*>(ws);
  int64_t* boff = reinterpret_cast<int64_t*>(ws + sizeof(int32_t) * kVBuckets);
  unsigned long long* cursor =
      reinterpret_cast<unsigned long long*>(ws + sizeof(int32_t) * kVBuckets + sizeof(int64_t) * (kVBuckets + 1));
  void* scan = ws + ((sizeof(int32_t) * kVBuckets + sizeof(int64_t) * (kVBuckets + 1) +
                      sizeof(unsigned long long) * kVBuckets + 15) & ~size_t(15));
  int rc = CB_OK;
  cudaError_t e = cudaSuccess;
  const unsigned g = grid_of(n, 256, h->num_sms);
  const unsigned wgrid = grid_of(n * 32, 256, h->num_sms);
  k_lower_count<<<g, 256, 0, s>>>(n, rp, col, low);
  if ((e = exclusive_scan_i32(low, grp, n, h->scan_ws, s, &h->launches)) == cudaSuccess &&
      (e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * kVBuckets, s)) == cudaSuccess) {
    k_vcount<<<wgrid, 256, 0, s>>>(n, rp, col, sh, hist);
    if ((e = exclusive_scan_i32(hist, boff, nb, scan, s, &h->launches)) == cudaSuccess) {
      k_vcursor<<<(nb + 255) / 256, 256, 0, s>>>(nb, boff, cursor);
      // the scratch holds row_ptr[n] int32: room for row_ptr[n] / 2 pairs,
      // exactly the entries above the diagonal of a symmetric graph
      const int64_t cap = h->nnz / 2;
      k_vpart<<<h->num_sms * 4, 256, 0, s>>>(n, rp, col, sh, cursor, reinterpret_cast<int2*>(grouped),
                                             static_cast<unsigned long long>(cap), h->err);
      k_vcheck<<<g, 256, 0, s>>>(n, rp, col, low, reinterpret_cast<const int2*>(grouped), boff, nb, grp, cap,
                                 h->err);
      e = cudaGetLastError();
      h->launches += 5;
    }
  }
  if (e != cudaSuccess) rc = cuda_fail(h, e, "validation");
  cudaFreeAsync(ws, s);
  h->dev_bytes -= static_cast<int64_t>(ws_bytes);
  return rc;
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

// Canonical pairs of the current step: id-space rows (unsorted), the count
// above the diagonal per row, and each row's upper part sorted into place.
int export_sorted_pairs(Graph* h, int32_t* pairs) {
  const int64_t n = h->n;
  if (n == 0) return CB_OK;
  int rc;
  const int spare = 1 - h->cur;
  if ((rc = invert_permutation(h, h->order[h->cur], h->pos_next))) return rc;
  if ((rc = relabel_rows(h, n, h->rp[h->cur], h->col[h->cur], h->pos_next, h->order[h->cur], h->rp_id,
                         h->col[spare])))
    return rc;
  int32_t* cnt = h->deg_next;      // free between super steps
  int64_t* off = h->rp[spare];
  cudaStream_t s = h->stream;
  const unsigned wgrid = grid_of(n * 32, 256, h->num_sms);
  k_count_above<<<wgrid, 256, 0, s>>>(n, h->rp_id, h->col[spare], cnt);
  CB_CUDA(h, cudaGetLastError());
  CB_CUDA(h, exclusive_scan_i32(cnt, off, n, h->scan_ws, s, &h->launches));
  AboveArgs a{n, h->rp_id, h->col[spare], cnt, off, h->segs, h->seg_of, pairs, h->err};
  k_above_warp<<<grid_of(n, 8, h->num_sms), 256, 0, s>>>(a);
  CB_CUDA(h, cudaGetLastError());
  h->launches += 2;
  if (h->maxdeg > kRowWarpMax) {
    constexpr int kMid = 2048;
    k_above_block<<<h->num_sms * 8, 256, kMid * 4, s>>>(a, kRowWarpMax, kMid, kMid, nullptr, 0);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    if (h->maxdeg > kMid) {
      int64_t slice = 0;
      int ctas = h->num_sms * 2;
      int32_t* gws = nullptr;
      if (h->maxdeg > kRowBlockSmem) {
        slice = next_pow2_host(h->maxdeg);
        const size_t budget = h->ws_slice * static_cast<size_t>(h->ws_ctas);
        if (budget < static_cast<size_t>(slice) * 4) return fail(h, CB_ENOMEM, "row workspace too small");
        ctas = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ctas, budget / (slice * 4))));
        gws = static_cast<int32_t*>(h->ws_global);
      }
      CB_CUDA(h, cudaFuncSetAttribute(k_above_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kRowBlockSmem * 4));
      k_above_block<<<ctas, 256, kRowBlockSmem * 4, s>>>(a, kMid, INT64_MAX, kRowBlockSmem, gws, slice);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
    }
  }
  return CB_OK;
}

}  // namespace cb
