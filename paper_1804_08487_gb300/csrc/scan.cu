// Device exclusive prefix sums (int32 or int64 input -> int64 output), used for
// CSR row offsets and bucket offsets.  Blocks of 256 threads x 8 items; block
// totals are scanned recursively.
#include "cb_internal.cuh"
#include "team.cuh"

namespace cb {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = kScanThreads * kScanItems;

template <class Tin>
__global__ void __launch_bounds__(kScanThreads) k_block_sums(const Tin* __restrict__ in, int64_t n,
                                                             int64_t* __restrict__ bsum) {
  __shared__ int64_t red[BlockTeam<kScanThreads>::kRedSlots];
  BlockTeam<kScanThreads> tm(red);
  const int64_t base = blockIdx.x * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < n) s += static_cast<int64_t>(in[base + j]);
  s = tm.sum(s);
  if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

template <class Tin>
__global__ void __launch_bounds__(kScanThreads) k_block_scan(const Tin* __restrict__ in, int64_t n,
                                                             const int64_t* __restrict__ boff,
                                                             int64_t* __restrict__ out) {
  __shared__ int64_t red[BlockTeam<kScanThreads>::kRedSlots];
  BlockTeam<kScanThreads> tm(red);
  const int64_t base = blockIdx.x * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = (base + j < n) ? static_cast<int64_t>(in[base + j]) : 0;
    s += v[j];
  }
  int64_t run = tm.exscan(s) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) {
      out[base + j] = run;
      run += v[j];
      if (base + j == n - 1) out[n] = run;
    }
  }
}

template <class Tin>
cudaError_t scan_rec(const Tin* in, int64_t* out, int64_t n, int64_t* ws, cudaStream_t s, int64_t* launches) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_block_scan<Tin><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  int64_t* bsum = ws;
  int64_t* boff = ws + nb;
  int64_t* rest = boff + nb + 1;
  k_block_sums<Tin><<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, bsum);
  if (launches) *launches += 2;
  cudaError_t e = scan_rec<int64_t>(bsum, boff, nb, rest, s, launches);
  if (e != cudaSuccess) return e;
  k_block_scan<Tin><<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, boff, out);
  return cudaGetLastError();
}

}  // namespace

size_t scan_ws_bytes(int64_t n) {
  size_t total = 0;
  while (n > kScanTile) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    total += static_cast<size_t>(2 * nb + 1);
    n = nb;
  }
  return (total + 16) * sizeof(int64_t);
}

cudaError_t exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s,
                               int64_t* launches) {
  return scan_rec<int32_t>(in, out, n, static_cast<int64_t*>(ws), s, launches);
}

}  // namespace cb
