// The permutation pi of a super step (Def. "Undirected Global Trade"): node x
// gets the key philox64(seed; x, 0, g, 0) and the nodes are ordered by
// (key, x).  Sorting is MSD-bucketed: a histogram of the top B key bits, a
// scatter of (key, x) into buckets, then one CTA sorts each bucket (about 512
// entries, keys are uniform) in shared memory by a counting sort on the 10
// key bits below the highest bit where the bucket's keys differ (about one
// key per bin; keys sharing a bin are ranked against each other).  A bucket
// above the shared memory cap is ranked by a slow global-memory fallback.
#include "cb_internal.cuh"
#include "philox.cuh"
#include "team.cuh"

#include <mutex>

namespace cb {

int bucket_bits(int64_t n) {
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= n) ++lg;
  return lg > 9 ? lg - 9 : 0;
}

namespace {

constexpr int kPermThreads = 256;

__device__ __forceinline__ uint32_t bucket_of(uint64_t key, int B) {
  return B == 0 ? 0u : static_cast<uint32_t>(key >> (64 - B));
}

// Where node keys come from: a handle's segment table (each segment at its
// device step + dg, or every segment at g_abs when use_abs), or one segment
// passed by value (segs == nullptr).
struct KeySrc {
  const Seg* segs;
  const int32_t* seg_of;
  Seg s0;
  uint32_t dg;
  int use_abs;
  uint32_t g_abs;
};

// Permutation key and bucket of node x.  A padding node gets the largest key.
__device__ __forceinline__ void key_of(const KeySrc& ks, int64_t x, uint64_t& key, uint32_t& bucket) {
  uint64_t seed;
  int64_t off, n, base;
  uint32_t g;
  int B;
  if (ks.segs) {
    const Seg* S = ks.segs + (ks.seg_of ? __ldg(ks.seg_of + x) : 0);
    seed = __ldg(&S->seed);
    off = __ldg(&S->off);
    n = __ldg(&S->n);
    base = __ldg(&S->bucket_base);
    g = ks.use_abs ? ks.g_abs : __ldg(&S->g) + ks.dg;
    B = __ldg(&S->B);
  } else {
    seed = ks.s0.seed;
    off = ks.s0.off;
    n = ks.s0.n;
    base = ks.s0.bucket_base;
    g = ks.use_abs ? ks.g_abs : ks.s0.g + ks.dg;
    B = ks.s0.B;
  }
  const int64_t l = x - off;
  key = l < n ? node_key(seed, static_cast<uint32_t>(l), g) : ~0ull;
  bucket = static_cast<uint32_t>(base) + bucket_of(key, B);
}

__global__ void k_perm_hist(int64_t n, KeySrc ks, int nb, int32_t* __restrict__ hist) {
  extern __shared__ int32_t sh[];
  const bool local = nb <= 4096;
  if (local) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    uint64_t k;
    uint32_t b;
    key_of(ks, x, k, b);
    if (local) atomicAdd(&sh[b], 1); else atomicAdd(&hist[b], 1);
  }
  if (local) {
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
  }
}

__global__ void k_perm_scatter(int64_t n, KeySrc ks, const int64_t* __restrict__ boff, int32_t* __restrict__ cursor,
                               uint64_t* __restrict__ bkey, int32_t* __restrict__ bid) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    uint64_t k;
    uint32_t b;
    key_of(ks, x, k, b);
    const int64_t slot = boff[b] + atomicAdd(&cursor[b], 1);
    bkey[slot] = k;
    bid[slot] = static_cast<int32_t>(x);
  }
}

// ------------------------------------------- relaxed global trade (no sort)
//
// Def. "Relaxed global trade" with a linear congruential map
// h(x) = (a x + b) mod p, p the smallest prime >= n: the nodes in order of
// h(x).  The image of [n] is Z_p minus the p - n values h takes on [n, p)
// (the gaps; p - n is below a few hundred for any n < 2^31), so node x sits
// at position h(x) - #{gaps below h(x)}, with no sort.  (a, b) come from
// Philox4x32-10 on counter (0, 0, g, 4): a = 1 + (r0r1 mod (p-1)),
// b = r2r3 mod p.

__device__ __forceinline__ uint64_t mulmod(uint64_t x, uint64_t y, uint64_t p) { return (x * y) % p; }

// One CTA: (a, b) of the step, the gap values h(x), n <= x < p, sorted into gaps[1..]
// (gaps[0] = their count).
__global__ void k_lcg_gaps(int64_t n, uint64_t p, KeySrc ks, uint64_t* __restrict__ ab, int64_t* __restrict__ gaps) {
  __shared__ int64_t sg[kMaxLcgGaps];
  const uint64_t seed = ks.segs ? ks.segs[0].seed : ks.s0.seed;
  const uint32_t g = ks.use_abs ? ks.g_abs : (ks.segs ? ks.segs[0].g : ks.s0.g) + ks.dg;
  const Philox4 r = philox4x32_10(0u, 0u, g, 4u, seed);
  const uint64_t a = 1 + (((static_cast<uint64_t>(r.w0) << 32) | r.w1) % (p - 1));
  const uint64_t b = ((static_cast<uint64_t>(r.w2) << 32) | r.w3) % p;
  const int ng = static_cast<int>(p - static_cast<uint64_t>(n));
  int P = 1;
  while (P < ng) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    sg[i] = i < ng ? static_cast<int64_t>((mulmod(a, static_cast<uint64_t>(n + i), p) + b) % p) : INT64_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const int64_t x = sg[i], y = sg[l];
          if ((x > y) == ((i & k) == 0)) { sg[i] = y; sg[l] = x; }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < ng; i += blockDim.x) gaps[1 + i] = sg[i];
  if (threadIdx.x == 0) {
    gaps[0] = ng;
    ab[0] = a;
    ab[1] = b;
  }
}

// Node x goes to position h(x) - #{gaps < h(x)}.
__global__ void k_lcg_positions(int64_t n, uint64_t p, const uint64_t* __restrict__ ab,
                                const int64_t* __restrict__ gaps, int32_t* __restrict__ order,
                                int32_t* __restrict__ pos) {
  __shared__ int64_t sg[kMaxLcgGaps];
  const int ng = static_cast<int>(gaps[0]);
  for (int i = threadIdx.x; i < ng; i += blockDim.x) sg[i] = gaps[1 + i];
  __syncthreads();
  const uint64_t a = ab[0], b = ab[1];
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t y = static_cast<int64_t>((mulmod(a, static_cast<uint64_t>(x), p) + b) % p);
    int lo = 0, hi = ng;   // gaps below y
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sg[mid] < y) lo = mid + 1; else hi = mid;
    }
    const int64_t q = y - lo;
    order[q] = static_cast<int32_t>(x);
    if (pos) pos[x] = static_cast<int32_t>(q);
  }
}

__device__ __forceinline__ bool pair_less(uint64_t ka, int32_t ia, uint64_t kb, int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// One CTA per bucket.  A bucket's keys agree on their leading bits and are
// uniform below them, so a counting sort on the kSubBits bits below the
// highest bit where they differ leaves about one key per bin for buckets of
// up to ~kSubBins keys (keys agree above that bit, so the digit orders them);
// keys sharing a bin are ranked by comparing (key, id) with each other.
constexpr int kSubBits = 10;
constexpr int kSubBins = 1 << kSubBits;
// dynamic shared memory: keys, ids, bin starts (+1), bin cursors, and each
// bin slot's element
size_t bucket_smem_bytes(int cap_pow2) {
  return static_cast<size_t>(cap_pow2) * (sizeof(uint64_t) + sizeof(int32_t) + sizeof(uint16_t)) +
         (2 * kSubBins + 1) * sizeof(int32_t);
}
__global__ void __launch_bounds__(kPermThreads) k_bucket_sort(
    int nb, const int64_t* __restrict__ boff, const uint64_t* __restrict__ bkey,
    const int32_t* __restrict__ bid, int cap, int32_t* __restrict__ order,
    int32_t* __restrict__ pos, int32_t* __restrict__ overflow, int cap_pow2) {
  extern __shared__ uint64_t shk[];
  int32_t* shi = reinterpret_cast<int32_t*>(shk + cap_pow2);
  int32_t* bstart = shi + cap_pow2;        // kSubBins + 1
  int32_t* bcur = bstart + kSubBins + 1;   // kSubBins
  uint16_t* slot = reinterpret_cast<uint16_t*>(bcur + kSubBins);   // cap_pow2
  __shared__ unsigned long long s_or, s_and;
  __shared__ int wsum[kPermThreads / 32];
  constexpr int kPer = kSubBins / kPermThreads;   // bins per thread in the scan
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t o = boff[b];
    const int64_t bs = boff[b + 1] - o;
    const int s = static_cast<int>(bs < int64_t(cap) + 1 ? bs : int64_t(cap) + 1);
    if (s > cap) {
      if (threadIdx.x == 0) overflow[1 + atomicAdd(&overflow[0], 1)] = b;
      continue;
    }
    if (s == 0) continue;
    if (threadIdx.x == 0) {
      s_or = 0ull;
      s_and = ~0ull;
    }
    for (int i = threadIdx.x; i < kSubBins; i += kPermThreads) bcur[i] = 0;
    __syncthreads();
    unsigned long long lor = 0ull, land = ~0ull;
    for (int i = threadIdx.x; i < s; i += kPermThreads) {
      const uint64_t k = bkey[o + i];
      shk[i] = k;
      shi[i] = bid[o + i];
      lor |= k;
      land &= k;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      lor |= __shfl_xor_sync(0xffffffffu, lor, off);
      land &= __shfl_xor_sync(0xffffffffu, land, off);
    }
    if (lane == 0) {
      atomicOr(&s_or, lor);
      atomicAnd(&s_and, land);
    }
    __syncthreads();
    const uint64_t diff = s_or ^ s_and;            // the bits where the bucket's keys differ
    const int top = diff ? 63 - __clzll(static_cast<long long>(diff)) : 0;
    const int sh = top + 1 > kSubBits ? top + 1 - kSubBits : 0;
    for (int i = threadIdx.x; i < s; i += kPermThreads)
      atomicAdd(&bcur[static_cast<int>(shk[i] >> sh) & (kSubBins - 1)], 1);
    __syncthreads();
    // exclusive scan of the bin counts: kPer consecutive bins per thread
    int local = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) local += bcur[threadIdx.x * kPer + q];
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int run = incl - local;
    for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int bi = threadIdx.x * kPer + q;
      const int c = bcur[bi];
      bstart[bi] = run;
      bcur[bi] = run;   // now the bin's cursor
      run += c;
    }
    if (threadIdx.x == 0) bstart[kSubBins] = s;
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kPermThreads)
      slot[atomicAdd(&bcur[static_cast<int>(shk[i] >> sh) & (kSubBins - 1)], 1)] = static_cast<uint16_t>(i);
    __syncthreads();
    // rank within the bin: the bin's start plus the smaller (key, id) in it
    for (int i = threadIdx.x; i < s; i += kPermThreads) {
      const uint64_t ki = shk[i];
      const int32_t ii = shi[i];
      const int d = static_cast<int>(ki >> sh) & (kSubBins - 1);
      const int st = bstart[d], en = bstart[d + 1];
      int r = st;
      for (int q = st; q < en; ++q) {
        const int j = slot[q];
        r += (j != i && pair_less(shk[j], shi[j], ki, ii)) ? 1 : 0;
      }
      order[o + r] = ii;
      if (pos) pos[ii] = static_cast<int32_t>(o + r);
    }
    __syncthreads();
  }
}

// Fallback for buckets above the shared-memory cap: rank by counting.
__global__ void k_bucket_overflow(const int32_t* __restrict__ overflow, const int64_t* __restrict__ boff,
                                  const uint64_t* __restrict__ bkey, const int32_t* __restrict__ bid,
                                  int32_t* __restrict__ order, int32_t* __restrict__ pos) {
  const int cnt = overflow[0];
  for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
    const int b = overflow[1 + q];
    const int64_t o = boff[b], s = boff[b + 1] - o;
    for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
      const uint64_t ki = bkey[o + i];
      const int32_t ii = bid[o + i];
      int64_t r = 0;
      for (int64_t j = 0; j < s; ++j) r += pair_less(bkey[o + j], bid[o + j], ki, ii) ? 1 : 0;
      order[o + r] = ii;
      if (pos) pos[ii] = static_cast<int32_t>(o + r);
    }
  }
}

__global__ void k_prep_next(int64_t n, const int32_t* __restrict__ order_cur, const int32_t* __restrict__ order_next,
                            const int32_t* __restrict__ pos_next, const int32_t* __restrict__ deg_id,
                            int32_t* __restrict__ M, int32_t* __restrict__ Minv, int32_t* __restrict__ deg_next) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
    const int32_t q = pos_next[order_cur[p]];
    M[p] = q;
    Minv[q] = static_cast<int32_t>(p);
    deg_next[p] = deg_id[order_next[p]];
  }
}

struct PermWs {
  int32_t* hist;      // nb
  int32_t* cursor;    // nb
  int64_t* boff;      // nb + 1
  int32_t* overflow;  // nb + 1
  uint64_t* bkey;     // n
  int32_t* bid;       // n
  void* scan;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

PermWs carve(void* base, int64_t n, int64_t nb) {
  char* p = static_cast<char*>(base);
  PermWs w;
  w.hist = reinterpret_cast<int32_t*>(p); p += align_up(sizeof(int32_t) * nb);
  w.cursor = reinterpret_cast<int32_t*>(p); p += align_up(sizeof(int32_t) * nb);
  w.boff = reinterpret_cast<int64_t*>(p); p += align_up(sizeof(int64_t) * (nb + 1));
  w.overflow = reinterpret_cast<int32_t*>(p); p += align_up(sizeof(int32_t) * (nb + 1));
  w.bkey = reinterpret_cast<uint64_t*>(p); p += align_up(sizeof(uint64_t) * n);
  w.bid = reinterpret_cast<int32_t*>(p); p += align_up(sizeof(int32_t) * n);
  w.scan = p;
  return w;
}

unsigned grid_for(int64_t work, int threads, int num_sms) {
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = int64_t(num_sms) * 16;
  return static_cast<unsigned>(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

size_t perm_ws_bytes(int64_t n, int64_t nb) {
  return align_up(sizeof(int32_t) * nb) * 2 + align_up(sizeof(int64_t) * (nb + 1)) +
         align_up(sizeof(int32_t) * (nb + 1)) + align_up(sizeof(uint64_t) * n) +
         align_up(sizeof(int32_t) * n) + scan_ws_bytes(nb + 1) + 256;
}

// The bucket sort's shared memory for the largest "bucket_cap" (set once,
// outside any stream capture).
int init_perm_kernels(Graph* h) {
  CB_CUDA(h, cudaFuncSetAttribute(k_bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(bucket_smem_bytes(kBucketCapMax))));
  return CB_OK;
}

int compute_permutation(Graph* h, uint32_t dg, int64_t g_abs, int32_t* order_out, int32_t* pos_out) {
  const int64_t n = h->n;
  if (n == 0) return CB_OK;
  if (h->relaxed) {
    KeySrc ks{};
    ks.segs = h->segs;
    ks.dg = dg;
    ks.use_abs = g_abs >= 0;
    ks.g_abs = static_cast<uint32_t>(g_abs < 0 ? 0 : g_abs);
    k_lcg_gaps<<<1, 256, 0, h->stream>>>(n, h->lcg_p, ks, h->lcg_ab, h->lcg_gaps);
    CB_CUDA(h, cudaGetLastError());
    k_lcg_positions<<<grid_for(n, kPermThreads, h->num_sms), kPermThreads, 0, h->stream>>>(n, h->lcg_p, h->lcg_ab,
                                                                                          h->lcg_gaps, order_out,
                                                                                          pos_out);
    CB_CUDA(h, cudaGetLastError());
    h->launches += 2;
    return CB_OK;
  }
  const int64_t nb = h->nbuckets;
  PermWs w = carve(h->sort_ws, n, nb);
  cudaStream_t s = h->stream;
  CB_CUDA(h, cudaMemsetAsync(w.hist, 0, sizeof(int32_t) * nb, s));
  CB_CUDA(h, cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * nb, s));
  CB_CUDA(h, cudaMemsetAsync(w.overflow, 0, sizeof(int32_t), s));
  KeySrc ks{};
  ks.segs = h->segs;
  ks.seg_of = h->seg_of;
  ks.dg = dg;
  ks.use_abs = g_abs >= 0;
  ks.g_abs = static_cast<uint32_t>(g_abs < 0 ? 0 : g_abs);
  const unsigned grid = grid_for(n, kPermThreads, h->num_sms);
  const size_t hsm = nb <= 4096 ? sizeof(int32_t) * nb : 0;
  k_perm_hist<<<grid, kPermThreads, hsm, s>>>(n, ks, static_cast<int>(nb), w.hist);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(w.hist, w.boff, nb, w.scan, s, &h->launches));
  k_perm_scatter<<<grid, kPermThreads, 0, s>>>(n, ks, w.boff, w.cursor, w.bkey, w.bid);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  const int cap = h->bucket_cap;
  int cap_pow2 = 1;
  while (cap_pow2 < cap) cap_pow2 <<= 1;
  const size_t ssm = bucket_smem_bytes(cap_pow2);
  const unsigned sgrid = static_cast<unsigned>(nb < h->num_sms * 8 ? nb : h->num_sms * 8);
  k_bucket_sort<<<sgrid, kPermThreads, ssm, s>>>(static_cast<int>(nb), w.boff, w.bkey, w.bid, cap, order_out, pos_out,
                                                w.overflow, cap_pow2);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_bucket_overflow<<<64, kPermThreads, 0, s>>>(w.overflow, w.boff, w.bkey, w.bid, order_out, pos_out);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  return CB_OK;
}

int prepare_next(Graph* h) {
  const int nxt = 1 - h->cur;
  int rc = compute_permutation(h, 1, -1, h->order[nxt], h->pos_next);
  if (rc) return rc;
  const unsigned grid = grid_for(h->n, kPermThreads, h->num_sms);
  k_prep_next<<<grid, kPermThreads, 0, h->stream>>>(h->n, h->order[h->cur], h->order[nxt], h->pos_next,
                                                    h->deg_id, h->M, h->Minv, h->deg_next);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  CB_CUDA(h, exclusive_scan_i32(h->deg_next, h->rp[nxt], h->n, h->scan_ws, h->stream, &h->launches));
  return CB_OK;
}

}  // namespace cb

// ---------------------------------------------------------------------------
// The permutation without any allocation: same key sort, with its scratch in
// a static device array instead of memory owned by a handle.  For callers
// that may not allocate device memory themselves -- for example code running
// under a host framework that owns every device allocation, or a latency-
// critical loop where cudaMalloc could synchronise the device or fail.
namespace cb {
namespace {
constexpr int64_t kStaticPermMaxNodes = int64_t(1) << 20;   // largest n accepted
constexpr size_t kStaticPermBytes = size_t(13) << 20;       // >= perm_ws_bytes(2^20)
constexpr int kStaticPermMaxDevices = 64;
std::mutex g_static_perm_mu;
void* g_static_perm_ptr[kStaticPermMaxDevices] = {};
}  // namespace
}  // namespace cb

// Scratch of cb_permutation_static, shared by every call on a device and held
// by every device that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_static_perm_scratch[cb::kStaticPermBytes];

extern "C" int cb_permutation_static(int64_t n, uint64_t seed, uint64_t g, int32_t* order_out,
                                     void* cuda_stream) {
  using namespace cb;
  if (n < 0 || (n > 0 && !order_out)) return fail(nullptr, CB_EINVAL, "cb_permutation_static: bad n or order_out");
  if (n > kStaticPermMaxNodes)
    return fail(nullptr, CB_ESIZE, "cb_permutation_static: n exceeds the static scratch limit of 2^20 nodes");
  if (g >= 0xfffffffeull) return fail(nullptr, CB_ERANGE, "cb_permutation_static: step too large");
  if (perm_ws_bytes(kStaticPermMaxNodes, int64_t(1) << bucket_bits(kStaticPermMaxNodes)) > kStaticPermBytes)
    return fail(nullptr, CB_ECHECK, "cb_permutation_static: static scratch smaller than its limit needs");
  if (n == 0) return CB_OK;
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kStaticPermMaxDevices) return fail(nullptr, CB_EINVAL, "cb_permutation_static: device index");
  void* base = nullptr;
  {
    // once per device, with that device current: the device address of the scratch
    std::lock_guard<std::mutex> lock(g_static_perm_mu);
    if (!g_static_perm_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_perm_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
      g_static_perm_ptr[dev] = p;
    }
    base = g_static_perm_ptr[dev];
  }
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int B = bucket_bits(n);
  const int nb = 1 << B;
  PermWs w = carve(base, n, nb);
  // the scratch keeps the previous call's contents: clear the counters
  if ((e = cudaMemsetAsync(w.hist, 0, sizeof(int32_t) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.overflow, 0, sizeof(int32_t), s)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaMemsetAsync");
  const unsigned grid = grid_for(n, kPermThreads, num_sms);
  const size_t hsm = nb <= 4096 ? sizeof(int32_t) * nb : 0;
  KeySrc ks{};
  ks.s0.seed = seed;
  ks.s0.n = n;
  ks.s0.span = n;
  ks.s0.B = B;
  ks.use_abs = 1;
  ks.g_abs = static_cast<uint32_t>(g);
  k_perm_hist<<<grid, kPermThreads, hsm, s>>>(n, ks, nb, w.hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "k_perm_hist");
  if ((e = exclusive_scan_i32(w.hist, w.boff, nb, w.scan, s)) != cudaSuccess) return cuda_fail(nullptr, e, "scan");
  k_perm_scatter<<<grid, kPermThreads, 0, s>>>(n, ks, w.boff, w.cursor, w.bkey, w.bid);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "k_perm_scatter");
  const int cap = 2048;
  const size_t ssm = bucket_smem_bytes(cap);
  const unsigned sgrid = static_cast<unsigned>(nb < num_sms * 8 ? nb : num_sms * 8);
  k_bucket_sort<<<sgrid, kPermThreads, ssm, s>>>(nb, w.boff, w.bkey, w.bid, cap, order_out, nullptr, w.overflow, cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "k_bucket_sort");
  k_bucket_overflow<<<64, kPermThreads, 0, s>>>(w.overflow, w.boff, w.bkey, w.bid, order_out, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "k_bucket_overflow");
  return CB_OK;
}
