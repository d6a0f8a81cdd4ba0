// Seeded input graphs on the device: PLD([a,b), gamma) degree sequences
// (Section 2, "Randomisation and Distributions") realised by Havel-Hakimi
// (Section 5.2: the graphs of the runtime experiments).  The results are
// byte-identical to the host generator that tests and benchmarks use (same
// SplitMix64 draws, same inverse-CDF table built in the same order with
// correctly rounded IEEE operations, same Havel-Hakimi tie order).
//
// Degree sampling is one independent draw per node.  Havel-Hakimi is a
// sequential greedy: each step takes the node of largest residual degree d
// and joins it to the next d nodes of the residual order, which that step
// changes.  Here one warp runs the steps over the order kept in residual
// buckets (consecutive positions with equal residual degree); a step's d
// connections, its block swap inside the last bucket it reaches and its
// emitted edges are spread over the lanes.  The edges then become a CSR with
// sorted rows in parallel.
#include <cmath>

#include "cb_internal.cuh"

namespace cb {
namespace {

// ---- the generator's draws and series (the host generator's, on the device)

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm_unif(uint64_t seed, uint64_t stream, uint64_t i) {
  const uint64_t base = sm_mix(seed + stream * 0x632be59bd9b4e019ULL + 0x9e3779b97f4a7c15ULL);
  const uint64_t v = sm_mix(base + (i + 1) * 0x9e3779b97f4a7c15ULL);
  return __dmul_rn(static_cast<double>(v >> 11), 1.0 / 9007199254740992.0);
}
constexpr double kLn2 = 0.693147180559945309417232121458176568;
// ln x for x >= 1 (x = m 2^e, ln m = 2 atanh((m-1)/(m+1)))
__device__ double p_ln(double x) {
  int e = 0;
  while (x >= 2.0) { x = __dmul_rn(x, 0.5); e++; }
  if (x > 1.4142135623730951) { x = __dmul_rn(x, 0.5); e++; }
  const double s = __ddiv_rn(__dsub_rn(x, 1.0), __dadd_rn(x, 1.0)), s2 = __dmul_rn(s, s);
  double term = s, sum = 0.0;
  for (int k = 1; k < 80; k += 2) {
    sum = __dadd_rn(sum, __ddiv_rn(term, static_cast<double>(k)));
    term = __dmul_rn(term, s2);
  }
  return __dadd_rn(__dmul_rn(2.0, sum), __dmul_rn(static_cast<double>(e), kLn2));
}
// e^y for y <= 0 (y = q ln2 + r, Taylor series for e^r)
__device__ double p_exp_neg(double y) {
  int q = static_cast<int>(__ddiv_rn(y, kLn2));
  const double r = __dsub_rn(y, __dmul_rn(static_cast<double>(q), kLn2));
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; k++) {
    term = __dmul_rn(term, __ddiv_rn(r, static_cast<double>(k)));
    sum = __dadd_rn(sum, term);
  }
  for (; q < 0; q++) sum = __dmul_rn(sum, 0.5);
  return sum;
}
__device__ double p_pow_neg(int64_t k, double gamma) {
  const double dk = static_cast<double>(k);
  if (gamma == 2.0) return __ddiv_rn(1.0, __dmul_rn(dk, dk));
  if (gamma == 3.0) return __ddiv_rn(1.0, __dmul_rn(__dmul_rn(dk, dk), dk));
  return p_exp_neg(-__dmul_rn(gamma, p_ln(dk)));
}

// the cumulative table of PLD([a, a+K), gamma), in order (one thread)
__global__ void k_pld_cdf(int32_t a, int64_t K, double gamma, double* cdf) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double z = 0.0;
  for (int64_t j = 0; j < K; j++) {
    z = __dadd_rn(z, (a + j == 0) ? 0.0 : p_pow_neg(a + j, gamma));
    cdf[j] = z;
  }
}

// degree i: the smallest j with cdf[j] > u z, u the i-th draw of stream 0
__global__ void k_pld_draw(int64_t n, int32_t a, int64_t K, uint64_t seed, const double* __restrict__ cdf,
                           int32_t* __restrict__ deg, unsigned long long* __restrict__ sum) {
  const double z = cdf[K - 1];
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double u = __dmul_rn(sm_unif(seed, 0, static_cast<uint64_t>(i)), z);
    int64_t lo = 0, hi = K - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    deg[i] = static_cast<int32_t>(a + lo);
    local += static_cast<unsigned long long>(a + lo);
  }
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(sum, local);
}

// odd sum: one more on the last degree
__global__ void k_pld_fix(int64_t n, int32_t* deg, unsigned long long* sum) {
  if (n > 0 && (*sum & 1ull)) {
    deg[n - 1] += 1;
    *sum += 1;
  }
}

// ---- Havel-Hakimi

// per-degree counts and the largest degree; degrees outside [0, n) fail
__global__ void k_hh_count(int64_t n, const int32_t* __restrict__ deg, int64_t* __restrict__ cnt, int32_t* dmax,
                           int32_t* err) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t d = deg[i];
    if (d < 0 || d >= n) {
      atomicCAS(err, 0, 1);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + d), 1ull);
    atomicMax(dmax, d);
  }
}

// bucket starts, buckets laid out from residual D down to 0 (one thread)
__global__ void k_hh_buckets(int32_t D, const int64_t* __restrict__ cnt, int64_t* __restrict__ bs,
                             int64_t* __restrict__ cur) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  bs[D] = 0;
  for (int64_t r = D - 1; r >= 0; r--) bs[r] = bs[r + 1] + cnt[r + 1];
  for (int64_t r = 0; r <= D; r++) cur[r] = bs[r];
}

// the initial order: by degree (descending buckets), ties by id -- one warp
// per degree value r walks the ids in increasing order
__global__ void k_hh_order(int64_t n, int32_t D, const int32_t* __restrict__ deg, int64_t* __restrict__ cur,
                           int32_t* __restrict__ ord) {
  // stable scatter: ids in increasing order, one block of ids at a time
  const int lane = threadIdx.x & 31;
  for (int64_t b0 = 0; b0 < n; b0 += 32) {
    const int64_t i = b0 + lane;
    const int32_t d = i < n ? deg[i] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(grp) - 1;
    int64_t base = 0;
    if (lane == leader && d >= 0) {
      base = cur[d];
      cur[d] = base + __popc(grp);
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (d >= 0) ord[base + __popc(grp & ((1u << lane) - 1u))] = static_cast<int32_t>(i);
  }
}

// The greedy itself, one warp.  res: residual degrees; bs / cnt: bucket
// start and size per residual; edges: (x, y) pairs appended in step order.
// status[0] = 0 success, 1 not graphical; status[1] = pairs written.
__global__ void k_hh_steps(int64_t n, int32_t* __restrict__ ord, int32_t* __restrict__ res, int64_t* __restrict__ bs,
                           int64_t* __restrict__ cnt, int2* __restrict__ edges, int64_t* __restrict__ status) {
  const int lane = threadIdx.x;
  int64_t front = 0, epos = 0;
  int failed = 0;
  while (front < n) {
    const int32_t x = ord[front];
    const int32_t d = res[x];
    if (d == 0) break;   // everything left is exhausted
    // consume x
    if (lane == 0) {
      bs[d] += 1;
      cnt[d] -= 1;
      res[x] = 0;
    }
    __syncwarp();
    front += 1;
    if (front + d > n || res[ord[front + d - 1]] == 0) {
      failed = 1;
      break;
    }
    const int32_t r_top = res[ord[front]];
    const int32_t r_last = res[ord[front + d - 1]];
    const int64_t start = bs[r_last], c = cnt[r_last];
    const int64_t k = front + d - start;   // targets inside bucket r_last
    // the d connections
    for (int64_t i = lane; i < d; i += 32) {
      const int32_t y = ord[front + i];
      edges[epos + i] = make_int2(x, y);
      res[y] -= 1;
    }
    epos += d;
    __syncwarp();
    // the k decremented members of bucket r_last move to its end (the same
    // block swap as the host procedure)
    if (k < c) {
      const int64_t w = 2 * k <= c ? k : c - k;
      const int64_t o = 2 * k <= c ? c - k : k;
      for (int64_t i = lane; i < w; i += 32) {
        const int32_t t = ord[start + i];
        ord[start + i] = ord[start + o + i];
        ord[start + o + i] = t;
      }
    }
    __syncwarp();
    if (lane == 0) {
      const int64_t keep = c - k;
      bs[r_last - 1] = start + keep;
      cnt[r_last - 1] += k;
      if (r_top > r_last) {   // buckets r_last+1..r_top were fully decremented: relabel them down
        bs[r_last] = (cnt[r_last + 1] > 0) ? bs[r_last + 1] : start;
        cnt[r_last] = cnt[r_last + 1] + keep;
        for (int64_t r = static_cast<int64_t>(r_last) + 2; r <= r_top; r++) {
          bs[r - 1] = bs[r];
          cnt[r - 1] = cnt[r];
        }
        cnt[r_top] = 0;
      } else {
        cnt[r_last] = keep;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    status[0] = failed;
    status[1] = epos;
  }
}

// every residual must be 0 at the end
__global__ void k_hh_residual(int64_t n, const int32_t* __restrict__ res, int64_t* status) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (res[i] != 0) status[0] = 1;
}

// the pairs into both rows
__global__ void k_hh_fill(int64_t m, const int2* __restrict__ edges, unsigned long long* __restrict__ fill,
                          int32_t* __restrict__ col) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
    const int2 p = edges[e];
    col[atomicAdd(fill + p.x, 1ull)] = p.y;
    col[atomicAdd(fill + p.y, 1ull)] = p.x;
  }
}

// rows sorted ascending: a CTA per row, a bitonic network in shared memory
// (rows of at most CAP entries; longer ones latch an error)
constexpr int kSortCap = 16384;
template <int CAP>
__global__ void k_sort_rows(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ col, int32_t* err) {
  extern __shared__ int32_t buf[];
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    const int64_t b = rp[r], len = rp[r + 1] - rp[r];
    if (len <= 1) continue;
    if (len > CAP) {
      if (threadIdx.x == 0) atomicCAS(err, 0, 2);   // longer than CAP
      continue;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) buf[i] = i < len ? col[b + i] : 0x7fffffff;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const int32_t x = buf[i], y = buf[l];
            const bool up = (i & kk) == 0;
            if ((x > y) == up) {
              buf[i] = y;
              buf[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) col[b + i] = buf[i];
    __syncthreads();
  }
}

}  // namespace
}  // namespace cb

using namespace cb;

extern "C" int cb_generate_pld(int64_t n, int32_t a, int32_t b, double gamma, uint64_t seed, int32_t* deg_out,
                               int64_t* sum_out, void* cuda_stream) {
  if (n < 0 || a < 0 || b <= a || (n > 0 && !deg_out) || !sum_out || !(gamma >= 1.0))
    return fail(nullptr, CB_EINVAL, "cb_generate_pld: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int64_t K = static_cast<int64_t>(b) - a;
  double* cdf = nullptr;
  unsigned long long* sum = nullptr;
  cudaError_t e = cudaMallocAsync(&cdf, sizeof(double) * K, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&sum, sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    if (cdf) cudaFreeAsync(cdf, s);
    return fail(nullptr, CB_ENOMEM, "cb_generate_pld: device allocation failed");
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s);
  k_pld_cdf<<<1, 32, 0, s>>>(a, K, gamma, cdf);
  if (n > 0)
    k_pld_draw<<<static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8))), 256, 0, s>>>(
        n, a, K, seed, cdf, deg_out, sum);
  k_pld_fix<<<1, 1, 0, s>>>(n, deg_out, sum);
  unsigned long long hsum = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hsum, sum, sizeof(hsum), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(cdf, s);
  cudaFreeAsync(sum, s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cb_generate_pld");
  *sum_out = static_cast<int64_t>(hsum);
  return CB_OK;
}

extern "C" int cb_generate_hh(int64_t n, const int32_t* deg, int64_t* row_ptr, int32_t* col, int64_t* m_out,
                              void* cuda_stream) {
  if (n < 0 || (n > 0 && (!deg || !row_ptr)) || !m_out) return fail(nullptr, CB_EINVAL, "cb_generate_hh: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  *m_out = 0;
  if (n == 0) return CB_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8)));
  // degrees: sum, largest, row offsets (host round trips are fine here)
  int32_t* err = nullptr;
  int64_t* status = nullptr;
  cudaError_t e = cudaMallocAsync(&err, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&status, 2 * sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), s);
  void* scan = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&scan, scan_ws_bytes(n + 1), s);
  if (e == cudaSuccess) e = exclusive_scan_i32(deg, row_ptr, n, scan, s);
  int64_t S = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&S, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  int64_t* cnt = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&cnt, sizeof(int64_t) * (n + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 2), s);
  if (e == cudaSuccess) k_hh_count<<<grid, 256, 0, s>>>(n, deg, cnt, err + 1, err);
  int32_t herr[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int32_t D = herr[1];
  int rc = CB_OK;
  int32_t *ord = nullptr, *res = nullptr;
  int64_t *bs = nullptr, *cur = nullptr;
  int2* edges = nullptr;
  if (e == cudaSuccess && (herr[0] || (S & 1))) {
    rc = -1;
  } else if (e == cudaSuccess && S > 0) {
    e = cudaMallocAsync(&ord, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&res, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&bs, sizeof(int64_t) * (D + 2), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&cur, sizeof(int64_t) * (n + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&edges, sizeof(int2) * (S / 2), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, deg, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
      k_hh_buckets<<<1, 1, 0, s>>>(D, cnt, bs, cur);
      k_hh_order<<<1, 32, 0, s>>>(n, D, deg, cur, ord);
      k_hh_steps<<<1, 32, 0, s>>>(n, ord, res, bs, cnt, edges, status);
      k_hh_residual<<<grid, 256, 0, s>>>(n, res, status);
      e = cudaGetLastError();
    }
    int64_t hs[2] = {1, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (hs[0] || hs[1] != S / 2)) rc = -1;
    if (e == cudaSuccess && rc == CB_OK) {
      // CSR: both directions of every pair (next free slot of each row in
      // `cur`), then sorted rows
      unsigned long long* fill = reinterpret_cast<unsigned long long*>(cur);
      e = cudaMemcpyAsync(fill, row_ptr, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sort_rows<kSortCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     static_cast<int>(sizeof(int32_t) * kSortCap));
      if (e == cudaSuccess) {
        k_hh_fill<<<grid, 256, 0, s>>>(S / 2, edges, fill, col);
        k_sort_rows<kSortCap><<<static_cast<unsigned>(std::min<int64_t>(n, int64_t(sms) * 4)), 512,
                                sizeof(int32_t) * kSortCap, s>>>(n, row_ptr, col, err);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess && herr[0]) rc = CB_ESIZE;
    }
  }
  for (void* p : {static_cast<void*>(ord), static_cast<void*>(res), static_cast<void*>(bs), static_cast<void*>(cur),
                  static_cast<void*>(edges), static_cast<void*>(cnt), scan, static_cast<void*>(err),
                  static_cast<void*>(status)})
    if (p) cudaFreeAsync(p, s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cb_generate_hh");
  if (rc == -1) return fail(nullptr, CB_EINVAL, "cb_generate_hh: degree sequence is not graphical");
  if (rc == CB_ESIZE) return fail(nullptr, CB_ESIZE, "cb_generate_hh: a row longer than 16384 entries");
  *m_out = S / 2;
  return CB_OK;
}
