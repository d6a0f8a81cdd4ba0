// Cooperative "teams" working on one trade or one row: part of a warp (8 or
// 16 lanes, LaneTeam), a warp (WarpTeam), part of a CTA (64 to 512 threads
// with a named barrier, SubTeam) or a whole CTA (BlockTeam).
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

// W consecutive lanes of a warp (W = 8 or 16): a warp holds 32 / W such
// teams, each on its own trade.  Synchronisation and shuffles name only the
// team's lanes, so teams that diverge (different trip counts, an early
// return) never wait for each other; while they run the same instructions,
// one warp instruction serves all of them.
template <int W>
struct LaneTeam {
  static_assert(W == 8 || W == 16, "lane teams of 8 or 16 lanes");
  static constexpr int N = W;
  int rank;
  unsigned mask;
  __device__ __forceinline__ LaneTeam()
      : rank(threadIdx.x & (W - 1)), mask(((1u << W) - 1u) << ((threadIdx.x & 31) & ~(W - 1))) {}
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
  __device__ __forceinline__ bool any(bool p) const { return __any_sync(mask, p); }
  __device__ __forceinline__ int64_t sum(int64_t v) const {
#pragma unroll
    for (int o = W / 2; o; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
    return v;
  }
  __device__ __forceinline__ int64_t exscan(int64_t v) const {
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
      const int64_t y = __shfl_up_sync(mask, x, o, W);
      if (rank >= o) x += y;
    }
    return x - v;
  }
  __device__ __forceinline__ uint64_t bcast(uint64_t v, int src) const { return __shfl_sync(mask, v, src, W); }
};

// A CTA of NT threads; `red` points at kRedSlots int64 slots of shared memory.
// Reductions take one barrier: warp partials go to one of two buffers in
// turn, and every warp combines them itself.  A buffer is written again only
// two calls later, after the middle call's barrier, when every thread has read
// it.  Every thread must make the same sequence of calls.
template <int NT>
struct BlockTeam {
  static constexpr int N = NT;
  static constexpr int NW = NT / 32;
  static constexpr int kRedSlots = 2 * NW;
  int rank;
  int buf;
  int64_t* red;
  __device__ __forceinline__ BlockTeam(int64_t* r) : rank(threadIdx.x), buf(0), red(r) {}
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p); }
  __device__ int64_t sum(int64_t v) {
    const int lane = rank & 31;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    int64_t* part = red + buf * NW;
    if (lane == 0) part[rank >> 5] = v;
    __syncthreads();
    buf ^= 1;
    int64_t x = lane < NW ? part[lane] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
  }
  __device__ int64_t exscan(int64_t v) {
    const int lane = rank & 31, w = rank >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    int64_t* part = red + buf * NW;
    if (lane == 31) part[w] = x;
    __syncthreads();
    buf ^= 1;
    // warps before w, summed across the lanes of this warp
    int64_t before = lane < w ? part[lane] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) before += __shfl_xor_sync(kFull, before, o);
    return x - v + before;
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

namespace cb {

// A team of NT threads (a multiple of 32) inside a larger CTA: threads
// [id NT, (id+1) NT) form team id and synchronise on named barrier id+1
// (barrier 0 stays with the whole CTA), so several teams of one CTA work on
// different trades independently.  `red` points at the team's kRedSlots
// int64 slots of shared memory; reductions take one barrier, as BlockTeam's.
template <int NT>
struct SubTeam {
  static constexpr int N = NT;
  static constexpr int NW = NT / 32;
  static constexpr int kRedSlots = 2 * NW;
  int rank;
  int bar;
  int buf;
  int64_t* red;
  __device__ __forceinline__ SubTeam(int64_t* r, int id) : rank(threadIdx.x % NT), bar(id + 1), buf(0), red(r) {}
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT) : "memory"); }
  __device__ __forceinline__ bool any(bool p) const {
    int r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n selp.s32 %0, 1, 0, o;\n}"
        : "=r"(r)
        : "r"(p ? 1 : 0), "r"(bar), "n"(NT)
        : "memory");
    return r != 0;
  }
  __device__ int64_t sum(int64_t v) {
    const int lane = rank & 31;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    int64_t* part = red + buf * NW;
    if (lane == 0) part[rank >> 5] = v;
    sync();
    buf ^= 1;
    int64_t x = lane < NW ? part[lane] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
  }
  __device__ int64_t exscan(int64_t v) {
    const int lane = rank & 31, w = rank >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    int64_t* part = red + buf * NW;
    if (lane == 31) part[w] = x;
    sync();
    buf ^= 1;
    int64_t before = lane < w ? part[lane] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) before += __shfl_xor_sync(kFull, before, o);
    return x - v + before;
  }
};

}  // namespace cb
