// Edge presence series and their autocorrelation (Section 5.1, "Mixing of
// Edge-Switching, Curveball and Global Curveball").
//
// With the "presence" option a handle keeps, for every node pair {a, b}
// (a < b, local ids) of every graph, one bit per recorded state: bit t of
// the pair's series is set when the edge exists after the t-th recorded super
// step (t = 0: the state when recording started).  cb_autocorr classifies each
// pair that ever occurred: for thinning k, the transitions of the k-thinned
// series (entries 0, k, 2k, ...) are fitted to an independent and to a
// first-order Markov model, and the edge counts as correlated when the
// Markov model fits better by the Bayesian information criterion,
// G^2 = 2 (L_Markov - L_independent) > ln N over its N transitions (the
// criterion is the reading of this library; the paper cites it without
// printing it).  A constant series, and one with fewer than two thinned
// transitions, counts as independent.
#include <cmath>
#include <vector>

#include "cb_internal.cuh"

namespace cb {

struct PresenceBufs {
  int64_t T = 0;             // super steps the record holds after its step 0
  int64_t t = 0;             // states recorded so far
  int64_t W = 0;             // 32-bit words per pair
  int64_t pairs = 0;         // pairs over every graph
  uint32_t* bits = nullptr;  // pairs x W
  int64_t* base = nullptr;   // device: first pair of each graph
  size_t bytes = 0;          // device bytes of bits and base
  std::vector<int64_t> hbase;
};

namespace {

__device__ __forceinline__ int64_t pair_index(int64_t n, int64_t a, int64_t b) {
  return a * n - a * (a + 1) / 2 + (b - a - 1);
}

// One warp per position: every entry (x, y) with x < y (local ids) sets
// bit t of its pair.
__global__ void k_presence(int64_t npos, const int32_t* __restrict__ order, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const Seg* __restrict__ segs,
                           const int32_t* __restrict__ seg_of, const int64_t* __restrict__ base, int64_t W,
                           int64_t t, uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t p = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; p < npos; p += warps) {
    const int g = seg_of ? seg_of[p] : 0;
    const int64_t off = segs[g].off, n = segs[g].n;
    const int64_t x = order[p] - off;
    for (int64_t e = rp[p] + lane; e < rp[p + 1]; e += 32) {
      const int64_t y = order[col[e]] - off;
      if (x < y && y < n) {
        const int64_t q = base[g] + pair_index(n, x, y);
        atomicOr(bits + q * W + (t >> 5), 1u << (t & 31));
      }
    }
  }
}

__device__ __forceinline__ double xlogy(double a, double b) { return a == 0.0 ? 0.0 : a * log(a / b); }

// One warp per pair of graph g: lane l classifies thinnings k = l + 1 and
// k = l + 33.  out[0..kmax) correlated pairs, out[64..64+kmax) decisions
// within 1e-9 of the boundary, out[128] pairs that occurred.
__global__ void k_autocorr(int64_t npairs, int64_t first, int64_t W, int64_t states, int kmax,
                           const uint32_t* __restrict__ bits, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long acc[129];
  for (int i = threadIdx.x; i < 129; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t q = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; q < npairs; q += warps) {
    const uint32_t* s = bits + (first + q) * W;
    bool any = false;
    for (int64_t i = lane; i < W; i += 32) any |= __ldg(s + i) != 0u;
    if (!__any_sync(0xffffffffu, any)) continue;
    if (lane == 0) atomicAdd(&acc[128], 1ull);
    for (int r = 0; r < 2; ++r) {
      const int k = lane + 1 + 32 * r;
      if (k > kmax) continue;
      // thinned entries x_0 .. x_N at steps 0, k, ..., N k
      const int64_t N = (states - 1) / k;
      if (N < 2) continue;
      int64_t ones_head = 0, ones_tail = 0, n11 = 0;   // ones among x_0..x_{N-1}, among x_1..x_N, pairs (1,1)
      int prev = static_cast<int>(__ldg(s) & 1u);
      for (int64_t j = 1; j <= N; ++j) {
        const int64_t st = j * k;
        const int cur = static_cast<int>((__ldg(s + (st >> 5)) >> (st & 31)) & 1u);
        ones_head += prev;
        ones_tail += cur;
        n11 += prev & cur;
        prev = cur;
      }
      const double n10 = static_cast<double>(ones_head - n11), n01 = static_cast<double>(ones_tail - n11);
      const double d11 = static_cast<double>(n11), dN = static_cast<double>(N);
      const double n00 = dN - d11 - n10 - n01;
      const double r0 = n00 + n01, r1 = n10 + n11;           // rows: x_{s-1} = 0, 1
      const double c0 = n00 + n10, c1 = n01 + n11;           // columns: x_s = 0, 1
      const double l1 = xlogy(n00, r0) + xlogy(n01, r0) + xlogy(n10, r1) + xlogy(d11, r1);
      const double l0 = xlogy(c0, dN) + xlogy(c1, dN);
      const double m = 2.0 * (l1 - l0) - log(dN);
      if (m > 0.0) atomicAdd(&acc[k - 1], 1ull);
      if (fabs(m) < 1e-9) atomicAdd(&acc[64 + k - 1], 1ull);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 129; i += blockDim.x)
    if (acc[i]) atomicAdd(&out[i], acc[i]);
}

}  // namespace

void free_presence(Graph* h) {
  if (!h->pres) return;
  if (h->pres->bits) cudaFreeAsync(h->pres->bits, h->stream);
  if (h->pres->base) cudaFreeAsync(h->pres->base, h->stream);
  h->dev_bytes -= static_cast<int64_t>(h->pres->bytes);
  delete h->pres;
  h->pres = nullptr;
}

int record_presence(Graph* h) {
  PresenceBufs* b = h->pres;
  if (!b || b->t > b->T) return CB_OK;   // off, or full
  if (h->n > 0) {
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>((h->n + 7) / 8, int64_t(h->num_sms) * 16));
    k_presence<<<grid, 256, 0, h->stream>>>(h->n, h->order[h->cur], h->rp[h->cur], h->col[h->cur], h->segs,
                                           h->seg_of, b->base, b->W, b->t, b->bits);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  }
  b->t += 1;
  return CB_OK;
}

int set_presence(Graph* h, int64_t T) {
  free_presence(h);
  if (T == 0) return CB_OK;
  PresenceBufs* b = new (std::nothrow) PresenceBufs;
  if (!b) return fail(h, CB_ENOMEM, "host allocation failed");
  b->T = T;
  b->W = (T + 1 + 31) / 32;
  b->hbase.resize(h->nseg);
  int64_t pairs = 0;
  for (int g = 0; g < h->nseg; ++g) {
    b->hbase[g] = pairs;
    const int64_t n = h->hsegs[g].n;
    pairs += n * (n - 1) / 2;
  }
  b->pairs = pairs;
  const double bytes = static_cast<double>(pairs) * static_cast<double>(b->W) * 4.0;
  if (bytes > 64e9) {
    delete b;
    return fail(h, CB_EINVAL, "presence record above 64 GB (pairs x steps too large)");
  }
  const size_t nbits = std::max<size_t>(static_cast<size_t>(bytes), 4), nbase = sizeof(int64_t) * h->nseg;
  void* p = nullptr;
  void* q = nullptr;
  if (dev_alloc(h, &p, nbits)) {
    delete b;
    return fail(h, CB_ENOMEM, "device allocation failed (presence record)");
  }
  if (dev_alloc(h, &q, nbase)) {
    cudaFreeAsync(p, h->stream);
    h->dev_bytes -= static_cast<int64_t>(nbits);
    delete b;
    return fail(h, CB_ENOMEM, "device allocation failed (presence record)");
  }
  b->bits = static_cast<uint32_t*>(p);
  b->base = static_cast<int64_t*>(q);
  b->bytes = nbits + nbase;
  h->pres = b;
  CB_CUDA(h, cudaMemsetAsync(b->bits, 0, static_cast<size_t>(bytes), h->stream));
  CB_CUDA(h, cudaMemcpyAsync(b->base, b->hbase.data(), sizeof(int64_t) * h->nseg, cudaMemcpyHostToDevice,
                             h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));   // hbase is read by the copy
  return record_presence(h);                       // step 0: the current state
}

}  // namespace cb

extern "C" int cb_autocorr(cb_handle h, int32_t graph, int32_t kmax, int64_t* correlated, int64_t* near_ties,
                           int64_t* occurring, int64_t* states) {
  using namespace cb;
  if (!h || kmax < 1 || kmax > 64 || !correlated) return fail(h, CB_EINVAL, "bad argument (kmax in [1, 64])");
  if (!h->pres) return fail(h, CB_EINVAL, "no presence record (set the \"presence\" option first)");
  if (graph < -1 || graph >= h->nseg) return fail(h, CB_EINVAL, "graph index out of range");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  PresenceBufs* b = h->pres;
  const int64_t used = std::min(b->t, b->T + 1);
  unsigned long long* d = nullptr;
  if (dev_alloc(h, reinterpret_cast<void**>(&d), 129 * sizeof(unsigned long long)))
    return fail(h, CB_ENOMEM, "device allocation failed");
  CB_CUDA(h, cudaMemsetAsync(d, 0, 129 * sizeof(unsigned long long), h->stream));
  const int g0 = graph < 0 ? 0 : graph, g1 = graph < 0 ? h->nseg : graph + 1;
  for (int g = g0; g < g1; ++g) {
    const int64_t n = h->hsegs[g].n, np = n * (n - 1) / 2;
    if (np == 0) continue;
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>((np + 7) / 8, int64_t(h->num_sms) * 16));
    k_autocorr<<<grid, 256, 0, h->stream>>>(np, b->hbase[g], b->W, used, kmax, b->bits, d);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  }
  unsigned long long hv[129];
  CB_CUDA(h, cudaMemcpyAsync(hv, d, sizeof(hv), cudaMemcpyDeviceToHost, h->stream));
  CB_CUDA(h, cudaStreamSynchronize(h->stream));
  cudaFreeAsync(d, h->stream);
  h->dev_bytes -= 129 * sizeof(unsigned long long);
  for (int k = 0; k < kmax; ++k) {
    correlated[k] = static_cast<int64_t>(hv[k]);
    if (near_ties) near_ties[k] = static_cast<int64_t>(hv[64 + k]);
  }
  if (occurring) *occurring = static_cast<int64_t>(hv[128]);
  if (states) *states = used;
  return check_device_error(h);
}
