// Cooperative "teams": a warp or a whole CTA working on one trade or one row.
// The trade and row algorithms are written once against this interface; all
// members of a team must reach every team call (team-uniform control flow).
#pragma once
#include <cstdint>

namespace cb {

constexpr unsigned kFull = 0xffffffffu;

struct WarpTeam {
  static constexpr int N = 32;
  int rank;
  __device__ __forceinline__ WarpTeam() : rank(threadIdx.x & 31) {}
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool any(bool p) const { return __any_sync(kFull, p); }
  __device__ __forceinline__ int64_t sum(int64_t v) const {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
  }
  // exclusive prefix sum over ranks
  __device__ __forceinline__ int64_t exscan(int64_t v) const {
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, x, o);
      if (rank >= o) x += y;
    }
    return x - v;
  }
  // value held by member `src`
  __device__ __forceinline__ uint64_t bcast(uint64_t v, int src) const { return __shfl_sync(kFull, v, src); }
};

// A CTA of NT threads; `red` points at NT/32 + 2 int64 slots of shared memory.
template <int NT>
struct BlockTeam {
  static constexpr int N = NT;
  static constexpr int NW = NT / 32;
  int rank;
  int64_t* red;
  __device__ __forceinline__ BlockTeam(int64_t* r) : rank(threadIdx.x), red(r) {}
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p); }
  __device__ int64_t sum(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((rank & 31) == 0) red[rank >> 5] = v;
    __syncthreads();
    if (rank < 32) {
      int64_t x = rank < NW ? red[rank] : 0;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (rank == 0) red[NW] = x;
    }
    __syncthreads();
    const int64_t r = red[NW];
    __syncthreads();
    return r;
  }
  __device__ int64_t exscan(int64_t v) {
    const int lane = rank & 31, w = rank >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) red[w] = x;
    __syncthreads();
    if (rank < 32) {
      const int64_t t = rank < NW ? red[rank] : 0;
      int64_t s = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, s, o);
        if (rank >= o) s += y;
      }
      if (rank < NW) red[rank] = s - t;
    }
    __syncthreads();
    const int64_t r = x - v + red[w];
    __syncthreads();
    return r;
  }
};

// First index i in [0, len) with a[i] >= v (len if none).
template <class T>
__device__ __forceinline__ int lower_bound(const T* a, int len, T v) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// In-place ascending bitonic sort of a[0..P), P a power of two.
template <class Team, class T>
__device__ void team_bitonic_sort(Team& tm, T* a, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tm.rank; i < P; i += Team::N) {
        const int l = i ^ j;
        if (l > i) {
          const T x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { a[i] = y; a[l] = x; }
        }
      }
      tm.sync();
    }
  }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace cb
