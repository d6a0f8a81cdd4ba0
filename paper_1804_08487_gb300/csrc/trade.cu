// One global trade (Def. "Undirected Global Trade", Section 3.3) on the GPU.
//
// Layout: during super step g the graph is stored in position space -- row p
// holds the node at position p of the step's permutation and every entry is
// the neighbour's position (rows are sets; their order is not significant).
// Trade t owns rows 2t (u_t) and 2t+1 (v_t); the neighbour at position y
// belongs to trade y>>1.
//
// Edges joining trades s and t form a "block" of at most four edges.  A later
// trade t depends on an earlier trade s only when the block has at least two
// edges and one of t's nodes is adjacent to exactly one of s's nodes: only then
// can s's choice turn a disjoint neighbour of t into a common one or back.
// Everything else is independent, because each shuffle key belongs to an edge
// (its endpoints' positions at the start of the step), not to a node.  So a
// super step runs in two phases:
//
//  A. Every trade finds D = (A_u u A_v) \ (A_u n A_v) \ {u, v}
//     (Def. "Simple Undirected Trade"), keys its elements and publishes the
//     threshold (key, lo, hi) of its |A_{u-v}|-th smallest element: u keeps
//     exactly the elements at or below it (Fig. 2: u receives the first
//     |A_{u-v}| elements of sigma(D)).  A trade whose dependency has not
//     published yet is deferred to a later pass.  Per entry it stores one
//     byte: whether its own trade moves the edge, whether the far trade will
//     consider the edge, and the top six bits of the far trade's key for it.
//  B. Every trade writes its two rows for step g+1: each entry goes to u or v
//     by its own trade's bit; its far end is resolved against the far trade's
//     threshold (six-bit prefix first, the full key only on a prefix tie), and
//     positions are mapped to step g+1.
//
// Trades of at most `warp_max` entries run on one warp, up to `block_max` on a
// 256-thread CTA, larger ones on a 1024-thread CTA with up to `smem_max`
// entries in shared memory (a global-memory slice above that).
#include <algorithm>

#include "cb_internal.cuh"
#include "philox.cuh"
#include "team.cuh"

namespace cb {
namespace {

// meta bits per entry (phase A)
constexpr uint8_t kR = 1;       // entry sits in v's row
constexpr uint8_t kInD = 2;     // element of D_t
constexpr uint8_t kFlip = 4;    // trade t moves the edge to its other node
constexpr uint8_t kUV = 8;      // the edge {u_t, v_t}
// bits 4..7: initial block matrix: u~2s, u~2s+1, v~2s, v~2s+1

// hash slot: high word = position + 1 (0 = empty); low word flags: bit0 in u's
// row, bit1 in v's row, bit2 the u-row entry flips, bit3 the v-row entry flips
constexpr int kMedThreads = 256;
constexpr int kBigThreads = 1024;
constexpr int kWarpCapA = kWarpCapMax;   // entries per warp-path trade (static shared memory)

struct StepCtx {
  int64_t n, T;
  uint64_t seed;
  uint32_t g, stamp;
  const int64_t* rp;
  const int32_t* col;
  uint8_t* stash;
  uint64_t* thr_key;
  uint64_t* thr_tb;
  uint8_t* thr_top;
  uint32_t* done;
  int32_t* err;
  const int32_t* M;
  const int64_t* rp_next;
  int32_t* col_next;
  int32_t* def_out;
  int32_t* def_count;
  int32_t* gws_count;
};

struct SelOut {
  uint64_t key, tb;
  int32_t bin, below, cnt, pad;
};

struct TradeRows {
  int64_t b0;
  int du, dv;
  bool single;   // odd n: the untraded node at the last position
};

__device__ __forceinline__ TradeRows trade_rows(const StepCtx& c, int64_t t) {
  TradeRows r;
  r.b0 = c.rp[2 * t];
  const int64_t b1 = c.rp[2 * t + 1];
  r.single = (2 * t + 1 >= c.n);
  const int64_t b2 = r.single ? b1 : c.rp[2 * t + 2];
  r.du = static_cast<int>(b1 - r.b0);
  r.dv = static_cast<int>(b2 - b1);
  return r;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void latch(int32_t* err, int32_t code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ uint64_t tie_break(uint32_t lo, uint32_t hi) {
  return (static_cast<uint64_t>(lo) << 32) | hi;
}
// (key, tb) <= (tk, tt), lexicographic
__device__ __forceinline__ bool at_or_below(uint64_t key, uint64_t tb, uint64_t tk, uint64_t tt) {
  return key < tk || (key == tk && tb <= tt);
}

// Both trades' keys of the edge whose step-start positions are lo < hi.
struct EdgeKeys {
  uint64_t lo_side, hi_side;
};
__device__ __forceinline__ EdgeKeys edge_keys(uint64_t seed, uint32_t lo, uint32_t hi, uint32_t g) {
  const Philox4 r = philox4x32_10(lo, hi, g, 1u, seed);
  return {(static_cast<uint64_t>(r.w0) << 32) | r.w1, (static_cast<uint64_t>(r.w2) << 32) | r.w3};
}

// Does trade s send the edge (lo, hi) to its node at position 2s?  Full test.
__device__ __forceinline__ bool far_keeps_low(const StepCtx& c, int64_t s, uint32_t lo, uint32_t hi) {
  const uint64_t k = edge_key(c.seed, lo, hi, c.g, (lo >> 1) == static_cast<uint32_t>(s));
  return at_or_below(k, tie_break(lo, hi), __ldcg(c.thr_key + s), __ldcg(c.thr_tb + s));
}

// ------------------------------------------------------------ hash table

__device__ __forceinline__ uint32_t hslot(int32_t y, int lgH) {
  return (static_cast<uint32_t>(y) * 0x9E3779B1u) >> (32 - lgH);
}

__device__ __forceinline__ void h_insert(unsigned long long* h, int lgH, int32_t y, uint32_t bit) {
  const unsigned long long key = static_cast<unsigned long long>(static_cast<uint32_t>(y) + 1u) << 32;
  const uint32_t mask = (1u << lgH) - 1u;
  uint32_t s = hslot(y, lgH);
  for (;;) {
    unsigned long long cur = h[s];
    if ((cur >> 32) == 0) {
      const unsigned long long prev = atomicCAS(&h[s], 0ull, key | bit);
      if (prev == 0ull) return;
      cur = prev;
    }
    if ((cur >> 32) == (key >> 32)) {
      atomicOr(reinterpret_cast<unsigned int*>(&h[s]), bit);
      return;
    }
    s = (s + 1) & mask;
  }
}

// Slot of y, or -1 if y is not in the table.
__device__ __forceinline__ int h_find(const unsigned long long* h, int lgH, int32_t y) {
  const uint32_t want = static_cast<uint32_t>(y) + 1u;
  const uint32_t mask = (1u << lgH) - 1u;
  uint32_t s = hslot(y, lgH);
  for (;;) {
    const unsigned long long cur = h[s];
    const uint32_t k = static_cast<uint32_t>(cur >> 32);
    if (k == want) return static_cast<int>(s);
    if (k == 0) return -1;
    s = (s + 1) & mask;
  }
}
__device__ __forceinline__ uint32_t h_flags(const unsigned long long* h, int lgH, int32_t y) {
  const int s = h_find(h, lgH, y);
  return s < 0 ? 0u : static_cast<uint32_t>(h[s]);
}

// ---------------------------------------------------------- workspace

struct WsA {
  int32_t* y;                 // entries (positions)
  uint16_t* top;              // top 16 bits of the own key
  uint8_t* meta;
  uint8_t* far;               // top 6 bits of the far trade's key
  unsigned long long* hash;   // 2^lgH slots
  uint32_t* hist;             // 256 bins
  int lgH;
};

// table of at least twice the entries: probing always ends at an empty slot
__host__ __device__ inline int hash_lg(int L) {
  int lg = 1;
  while ((1 << lg) < 2 * L) ++lg;
  return lg;
}
__host__ __device__ inline size_t ws_a_bytes(int L) {
  const size_t L16 = (static_cast<size_t>(L) + 15) & ~size_t(15);
  return (size_t(1) << hash_lg(L)) * 8 + 1024 + L16 * 4 + L16 * 2 + L16 * 2 + 64;
}
__device__ inline WsA carve_a(void* base, int L) {
  const size_t L16 = (static_cast<size_t>(L) + 15) & ~size_t(15);
  char* p = static_cast<char*>(base);
  WsA w;
  w.lgH = hash_lg(L);
  w.hash = reinterpret_cast<unsigned long long*>(p); p += (size_t(1) << w.lgH) * 8;
  w.hist = reinterpret_cast<uint32_t*>(p); p += 1024;
  w.y = reinterpret_cast<int32_t*>(p); p += L16 * 4;
  w.top = reinterpret_cast<uint16_t*>(p); p += L16 * 2;
  w.meta = reinterpret_cast<uint8_t*>(p); p += L16;
  w.far = reinterpret_cast<uint8_t*>(p);
  return w;
}

__device__ __forceinline__ uint32_t lo_of(int64_t t2, uint8_t m, int32_t y) {
  return min(static_cast<uint32_t>(t2 + (m & kR)), static_cast<uint32_t>(y));
}
__device__ __forceinline__ uint32_t hi_of(int64_t t2, uint8_t m, int32_t y) {
  return max(static_cast<uint32_t>(t2 + (m & kR)), static_cast<uint32_t>(y));
}
__device__ __forceinline__ uint64_t own_key(const StepCtx& c, int64_t t, uint32_t lo, uint32_t hi) {
  return edge_key(c.seed, lo, hi, c.g, (lo >> 1) == static_cast<uint32_t>(t));
}

// One radix digit of the 16-bit key prefixes: histogram of (top >> shift) & 255
// over elements of D whose high byte equals `pre` (shift 0) or over all of D
// (shift 8), then the bin holding the kk-th element.
template <class Team>
__device__ void radix_digit(Team& tm, const WsA& w, int L, int shift, uint32_t pre, int kk, SelOut* out) {
  constexpr int BPM = (256 + Team::N - 1) / Team::N;
  for (int b = tm.rank; b < 256; b += Team::N) w.hist[b] = 0;
  tm.sync();
  for (int i = tm.rank; i < L; i += Team::N) {
    if (!(w.meta[i] & kInD)) continue;
    const uint32_t tp = w.top[i];
    if (shift == 8 || (tp >> 8) == pre) atomicAdd(&w.hist[(tp >> shift) & 255u], 1u);
  }
  tm.sync();
  const int b0 = tm.rank * BPM;
  int local = 0;
#pragma unroll
  for (int j = 0; j < BPM; ++j)
    if (b0 + j < 256) local += static_cast<int>(w.hist[b0 + j]);
  int below = static_cast<int>(tm.exscan(local));
#pragma unroll
  for (int j = 0; j < BPM; ++j) {
    const int b = b0 + j;
    if (b < 256) {
      const int hc = static_cast<int>(w.hist[b]);
      if (below < kk && kk <= below + hc) {
        out->bin = b;
        out->below = below;
        out->cnt = hc;
      }
      below += hc;
    }
  }
  tm.sync();
}

// k-th smallest (1-based) (key, lo, hi) over D: two radix digits on the stored
// 16-bit key prefixes, then the full keys of the remaining candidates.
template <class Team>
__device__ void select_kth(Team& tm, const StepCtx& c, const WsA& w, int L, int64_t t, int k, SelOut* out) {
  const int64_t t2 = 2 * t;
  radix_digit(tm, w, L, 8, 0, k, out);
  const uint32_t b1 = static_cast<uint32_t>(out->bin);
  int kk = k - out->below;
  const int cnt1 = out->cnt;
  tm.sync();
  uint32_t prefix = b1 << 8;
  bool full16 = false;
  if (cnt1 > 1) {
    radix_digit(tm, w, L, 0, b1, kk, out);
    prefix |= static_cast<uint32_t>(out->bin);
    kk -= out->below;
    tm.sync();
    full16 = true;
  }
  // candidates share the prefix; rank them by the full (key, lo, hi)
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    if (!(m & kInD)) continue;
    const uint32_t tp = w.top[i];
    if (full16 ? (tp != prefix) : ((tp >> 8) != b1)) continue;
    const uint32_t lo = lo_of(t2, m, w.y[i]), hi = hi_of(t2, m, w.y[i]);
    const uint64_t ki = own_key(c, t, lo, hi), tbi = tie_break(lo, hi);
    int r = 0;
    for (int j = 0; j < L; ++j) {
      const uint8_t mj = w.meta[j];
      if (j == i || !(mj & kInD)) continue;
      const uint32_t tj = w.top[j];
      if (full16 ? (tj != prefix) : ((tj >> 8) != b1)) continue;
      const uint32_t loj = lo_of(t2, mj, w.y[j]), hij = hi_of(t2, mj, w.y[j]);
      const uint64_t kj = own_key(c, t, loj, hij);
      r += (kj < ki || (kj == ki && tie_break(loj, hij) < tbi));
    }
    if (r == kk - 1) {
      out->key = ki;
      out->tb = tbi;
    }
  }
  tm.sync();
}

// Phase A for trade t.
template <class Team>
__device__ void phase_a(Team& tm, const StepCtx& c, int64_t t, const WsA& w, SelOut* sel) {
  const TradeRows tr = trade_rows(c, t);
  const int du = tr.du, dv = tr.dv, L = du + dv;
  const int H = 1 << w.lgH;
  for (int i = tm.rank; i < H; i += Team::N) w.hash[i] = 0ull;
  for (int i = tm.rank; i < L; i += Team::N) w.y[i] = __ldcg(c.col + tr.b0 + i);
  tm.sync();
  for (int i = tm.rank; i < L; i += Team::N) h_insert(w.hash, w.lgH, w.y[i], i >= du ? 2u : 1u);
  tm.sync();
  const int64_t t2 = 2 * t;
  bool defer = false, has_dependents = false;
  int cnt_a = 0;
  for (int i = tm.rank; i < L; i += Team::N) {
    const int r = i >= du;
    const int32_t yy = w.y[i];
    const int64_t s = yy >> 1;
    w.far[i] = 0;
    w.top[i] = 0;
    if (s == t) {
      w.meta[i] = static_cast<uint8_t>(r | kUV);
      continue;
    }
    const int32_t e0 = static_cast<int32_t>(2 * s);
    const uint32_t f0 = h_flags(w.hash, w.lgH, e0), f1 = h_flags(w.hash, w.lgH, e0 + 1);
    const int u0 = f0 & 1, v0 = (f0 >> 1) & 1, u1 = f1 & 1, v1 = (f1 >> 1) & 1;
    const int cu = u0 + u1, cv = v0 + v1;
    uint8_t m = static_cast<uint8_t>(r | (u0 << 4) | (u1 << 5) | (v0 << 6) | (v1 << 7));
    // a later trade s depends on t when it sees >= 2 block edges and one of
    // its own nodes holds exactly one of them
    if (!tr.single && s > t && s < c.T && cu + cv >= 2 && (u0 + v0 == 1 || u1 + v1 == 1)) has_dependents = true;
    int col_now = yy & 1;                            // s-node of this edge when t acts
    int other = r ? (col_now ? u1 : u0) : (col_now ? v1 : v0);
    const bool dep = !tr.single && s < t && (cu + cv >= 2) && (cu == 1 || cv == 1);
    if (dep) {
      if (ld_acquire(c.done + s) != c.stamp) {
        defer = true;
        continue;
      }
      // replay trade s's decisions on this block
      int m1[2][2] = {{0, 0}, {0, 0}};
      const int bits[2][2] = {{u0, u1}, {v0, v1}};
      const int cnt_row[2] = {cu, cv};
#pragma unroll
      for (int rho = 0; rho < 2; ++rho)
#pragma unroll
        for (int gam = 0; gam < 2; ++gam) {
          if (!bits[rho][gam]) continue;
          int g2 = gam;
          if (cnt_row[rho] == 1) {
            const uint32_t x = static_cast<uint32_t>(t2 + rho), y = static_cast<uint32_t>(e0 + gam);
            g2 = far_keeps_low(c, s, min(x, y), max(x, y)) ? 0 : 1;
          }
          m1[rho][g2] = 1;
          if (rho == r && gam == (yy & 1)) col_now = g2;
        }
      other = m1[1 - r][col_now];
    }
    {  // both trades' keys of this edge: own 16-bit prefix, far 6-bit prefix
      const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(yy);
      const uint32_t lo = min(x, y), hi = max(x, y);
      const EdgeKeys ek = edge_keys(c.seed, lo, hi, c.g);
      const bool lo_mine = (lo >> 1) == static_cast<uint32_t>(t);
      w.top[i] = static_cast<uint16_t>((lo_mine ? ek.lo_side : ek.hi_side) >> 48);
      w.far[i] = static_cast<uint8_t>((lo_mine ? ek.hi_side : ek.lo_side) >> 58);
    }
    if (!other && !tr.single) {
      m |= kInD;
      cnt_a += (r == 0);
    }
    w.meta[i] = m;
  }
  if (tm.any(defer)) {
    if (tm.rank == 0) c.def_out[atomicAdd(c.def_count, 1)] = static_cast<int32_t>(t);
    tm.sync();
    return;
  }
  const int a = static_cast<int>(tm.sum(cnt_a));
  const bool publish_fence = tm.any(has_dependents);
  uint64_t tk = 0, tt = 0;
  if (!tr.single && a > 0) {
    select_kth(tm, c, w, L, t, a, sel);
    tk = sel->key;
    tt = sel->tb;
  }
  const uint32_t tk16 = static_cast<uint32_t>(tk >> 48);
  // own decisions; flips are recorded in the hash for the far-side test
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    if (!(m & kInD)) continue;
    const int r = m & kR;
    const uint32_t tp = w.top[i];
    bool low;
    if (tp != tk16) {
      low = tp < tk16;
    } else {
      const uint32_t lo = lo_of(t2, m, w.y[i]), hi = hi_of(t2, m, w.y[i]);
      low = at_or_below(own_key(c, t, lo, hi), tie_break(lo, hi), tk, tt);
    }
    if ((low ? 0 : 1) != r) {
      w.meta[i] = m | kFlip;
      const int slot = h_find(w.hash, w.lgH, w.y[i]);
      atomicOr(reinterpret_cast<unsigned int*>(&w.hash[slot]), 4u << r);
    }
  }
  tm.sync();
  // will the far trade consider this edge?  Write the stash byte.
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    const int f = (m & kFlip) ? 1 : 0;
    int in_far = 0;
    if (!(m & kUV)) {
      const int r = m & kR;
      const int32_t yy = w.y[i];
      const int64_t s = yy >> 1;
      const int u0 = (m >> 4) & 1, u1 = (m >> 5) & 1, v0 = (m >> 6) & 1, v1 = (m >> 7) & 1;
      const int cr = r ? (v0 + v1) : (u0 + u1);
      if (tr.single || s < t) {
        in_far = (cr == 1);                 // trade s acted before t: initial block
      } else if (s < c.T) {
        if (u0 + u1 + v0 + v1 == 1) {
          in_far = 1;
        } else {                            // block after t's own decisions
          const int32_t e0 = static_cast<int32_t>(2 * s);
          const uint32_t f0 = h_flags(w.hash, w.lgH, e0), f1 = h_flags(w.hash, w.lgH, e0 + 1);
          const int myrow = r ^ f;
          int same = 0;
          // post-trade row of each block edge: u-row entries move to v when flipped, and back
          same += (f0 & 1) && (((f0 >> 2) & 1) == myrow);
          same += ((f0 >> 1) & 1) && ((1 ^ ((f0 >> 3) & 1)) == myrow);
          same += (f1 & 1) && (((f1 >> 2) & 1) == myrow);
          same += ((f1 >> 1) & 1) && ((1 ^ ((f1 >> 3) & 1)) == myrow);
          in_far = (same == 1);
        }
      }
    }
    c.stash[tr.b0 + i] = static_cast<uint8_t>(f | (in_far << 1) | (in_far ? (w.far[i] << 2) : 0));
  }
  if (tm.rank == 0 && !tr.single) {
    c.thr_key[t] = tk;
    c.thr_tb[t] = tt;
    c.thr_top[t] = static_cast<uint8_t>(tk >> 58);
    if (publish_fence) {
      __threadfence();
      st_release(c.done + t, c.stamp);
    }
  }
  tm.sync();
}

// Phase B for trade t: write its two rows in step g+1's layout (no workspace).
template <class Team>
__device__ void phase_b(Team& tm, const StepCtx& c, int64_t t) {
  const TradeRows tr = trade_rows(c, t);
  const int du = tr.du, dv = tr.dv, L = du + dv;
  const int64_t t2 = 2 * t;
  const int32_t pu = c.M[t2];
  const int64_t ou = c.rp_next[pu];
  int64_t ov = 0;
  bool bad = c.rp_next[pu + 1] - ou != du;
  if (dv > 0) {
    const int32_t pv = c.M[t2 + 1];
    ov = c.rp_next[pv];
    bad |= c.rp_next[pv + 1] - ov != dv;
  }
  if (bad) {
    if (tm.rank == 0) latch(c.err, kErrRowLength);
    return;
  }
  int64_t base0 = 0;   // entries already placed in u's new row
  for (int c0 = 0; c0 < L; c0 += Team::N) {
    const int i = c0 + tm.rank;
    int r2 = 2;        // 2: no entry
    int32_t out = 0;
    if (i < L) {
      const int r = i >= du;
      const int32_t yy = __ldcg(c.col + tr.b0 + i);
      const uint8_t st = c.stash[tr.b0 + i];
      r2 = r ^ (st & 1);
      int32_t y2 = yy;
      if (st & 2) {
        const int64_t s = yy >> 1;
        const uint32_t ft = st >> 2, tt = c.thr_top[s];
        bool low;
        if (ft != tt) {
          low = ft < tt;
        } else {
          const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(yy);
          low = far_keeps_low(c, s, min(x, y), max(x, y));
        }
        y2 = static_cast<int32_t>(2 * s) + (low ? 0 : 1);
      }
      out = c.M[y2];
    }
    const int is0 = (r2 == 0);
    const int64_t before0 = tm.exscan(is0);
    const int64_t in0 = tm.sum(is0);
    if (r2 == 0) {
      c.col_next[ou + base0 + before0] = out;
    } else if (r2 == 1) {
      c.col_next[ov + (static_cast<int64_t>(i) - (base0 + before0))] = out;
    }
    base0 += in0;
  }
  if (tm.rank == 0 && base0 != du) latch(c.err, kErrRowSide);
}

// ---------------------------------------------------------------- kernels

__global__ void k_classify(StepCtx c, int64_t ntasks, int warp_max, int block_max, int32_t* __restrict__ lw,
                           int32_t* __restrict__ lm, int32_t* __restrict__ lb, int32_t* __restrict__ counters) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < ntasks; t += int64_t(gridDim.x) * blockDim.x) {
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    if (L <= warp_max) lw[atomicAdd(&counters[0], 1)] = static_cast<int32_t>(t);
    else if (L <= block_max) lm[atomicAdd(&counters[1], 1)] = static_cast<int32_t>(t);
    else lb[atomicAdd(&counters[2], 1)] = static_cast<int32_t>(t);
  }
}

struct WarpWsA {
  unsigned long long hash[2 * kWarpCapA];
  uint32_t hist[256];
  int32_t y[kWarpCapA];
  uint16_t top[kWarpCapA];
  uint8_t meta[kWarpCapA];
  uint8_t far[kWarpCapA];
  SelOut sel;
};

__global__ void __launch_bounds__(256) k_phase_a_warp(StepCtx c, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ count) {
  __shared__ WarpWsA ws[kWarpsPerCta];
  WarpTeam tm;
  const int wid = threadIdx.x >> 5;
  const int64_t len = *count;
  for (int64_t q = blockIdx.x * int64_t(kWarpsPerCta) + wid; q < len; q += int64_t(gridDim.x) * kWarpsPerCta) {
    const int64_t t = list[q];
    const TradeRows tr = trade_rows(c, t);
    WsA w{ws[wid].y, ws[wid].top, ws[wid].meta, ws[wid].far, ws[wid].hash, ws[wid].hist, hash_lg(tr.du + tr.dv)};
    phase_a(tm, c, t, w, &ws[wid].sel);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_phase_a_block(StepCtx c, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ count, int smem_max, char* gws,
                                                      size_t slice) {
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[NT / 32 + 2];
  __shared__ SelOut sel;
  BlockTeam<NT> tm(red);
  const int64_t len = *count;
  for (int64_t q = blockIdx.x; q < len; q += gridDim.x) {
    const int64_t t = list[q];
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    char* base = sbuf;
    if (L > smem_max) {
      base = gws + slice * blockIdx.x;
      if (threadIdx.x == 0) atomicAdd(c.gws_count, 1);
    }
    phase_a(tm, c, t, carve_a(base, L), &sel);
  }
}

__global__ void __launch_bounds__(256) k_phase_b_warp(StepCtx c, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ count) {
  WarpTeam tm;
  const int wid = threadIdx.x >> 5;
  const int64_t len = *count;
  for (int64_t q = blockIdx.x * int64_t(kWarpsPerCta) + wid; q < len; q += int64_t(gridDim.x) * kWarpsPerCta)
    phase_b(tm, c, list[q]);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_phase_b_block(StepCtx c, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ count) {
  __shared__ int64_t red[NT / 32 + 2];
  BlockTeam<NT> tm(red);
  const int64_t len = *count;
  for (int64_t q = blockIdx.x; q < len; q += gridDim.x) phase_b(tm, c, list[q]);
}

}  // namespace

size_t trade_ws_slice_bytes(int64_t max_trade) {
  return (ws_a_bytes(static_cast<int>(max_trade)) + 255) & ~size_t(255);
}
size_t trade_smem_bytes(int entries) { return ws_a_bytes(entries); }

int super_step(Graph* h) {
  if (h->g >= 0xfffffffeull) return fail(h, CB_ERANGE, "super-step counter exhausted");
  cudaStream_t s = h->stream;
  const int nxt = 1 - h->cur;
  if (h->timing) CB_CUDA(h, cudaEventRecord(h->ev[0], s));
  int rc = prepare_next(h);
  if (rc) return rc;
  if (h->timing) CB_CUDA(h, cudaEventRecord(h->ev[1], s));
  StepCtx c;
  c.n = h->n;
  c.T = h->T;
  c.seed = h->seed;
  c.g = static_cast<uint32_t>(h->g);
  c.stamp = static_cast<uint32_t>(h->g + 1);
  c.rp = h->rp[h->cur];
  c.col = h->col[h->cur];
  c.stash = h->stash;
  c.thr_key = h->thr_key;
  c.thr_tb = h->thr_tb;
  c.thr_top = h->thr_top;
  c.done = h->done;
  c.err = h->err;
  c.M = h->M;
  c.rp_next = h->rp[nxt];
  c.col_next = h->col[nxt];
  int32_t* cnt = h->counters;   // [0..2] class lists, [3..8] deferred (ping-pong x class), [9] global slices
  c.gws_count = cnt + 9;
  CB_CUDA(h, cudaMemsetAsync(cnt, 0, 12 * sizeof(int32_t), s));
  const int64_t ntasks = h->ntasks;
  if (ntasks == 0) {
    h->cur = nxt;
    h->g += 1;
    return CB_OK;
  }
  const int warp_max = std::min(h->warp_max, kWarpCapA);
  const int block_max = std::max(h->block_max, warp_max);
  {
    const int64_t want = (ntasks + 255) / 256;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, h->num_sms * 8)));
    k_classify<<<grid, 256, 0, s>>>(c, ntasks, warp_max, block_max, h->list[0], h->list[1], h->list[2], cnt);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  }
  const size_t med_smem = ws_a_bytes(std::max(block_max, 1));
  const size_t big_smem = ws_a_bytes(std::max(h->smem_max, 1));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kMedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(med_smem)));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(big_smem)));
  const unsigned wgrid = static_cast<unsigned>(h->num_sms * 6);
  const unsigned mgrid = static_cast<unsigned>(h->num_sms * 4);
  const unsigned bgrid = static_cast<unsigned>(std::max(1, std::min(h->num_sms, h->ws_ctas)));
  char* gws = static_cast<char*>(h->ws_global);

  // phase A: one launch per class over its list, then passes over deferred trades
  auto launch_a = [&](const int32_t* const* lists, const int32_t* counts, int out) -> int {
    for (int k = 0; k < 3; ++k) {
      c.def_out = h->list_def[out][k];
      c.def_count = cnt + 3 + 3 * out + k;
      if (k == 0) {
        k_phase_a_warp<<<wgrid, 256, 0, s>>>(c, lists[0], counts + 0);
      } else if (k == 1) {
        k_phase_a_block<kMedThreads><<<mgrid, kMedThreads, med_smem, s>>>(c, lists[1], counts + 1, block_max, gws,
                                                                         h->ws_slice);
      } else {
        k_phase_a_block<kBigThreads><<<bgrid, kBigThreads, big_smem, s>>>(c, lists[2], counts + 2, h->smem_max, gws,
                                                                         h->ws_slice);
      }
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
    }
    return CB_OK;
  };
  const int32_t* first[3] = {h->list[0], h->list[1], h->list[2]};
  if ((rc = launch_a(first, cnt, 0))) return rc;
  int64_t passes = 1, deferred_total = 0;
  int in = 0;
  for (;;) {
    CB_CUDA(h, cudaMemcpyAsync(h->host_counters, cnt, 12 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CB_CUDA(h, cudaStreamSynchronize(s));
    const int32_t* hc = h->host_counters;
    if (passes == 1) {
      h->stats[2] = hc[0];
      h->stats[3] = hc[1] + hc[2];
    }
    const int64_t ndef = int64_t(hc[3 + 3 * in]) + hc[4 + 3 * in] + hc[5 + 3 * in];
    if (ndef == 0) break;
    deferred_total += ndef;
    if (passes > 100000) return fail(h, CB_ECHECK, "dependency resolution did not converge");
    const int out = 1 - in;
    CB_CUDA(h, cudaMemsetAsync(cnt + 3 + 3 * out, 0, 3 * sizeof(int32_t), s));
    const int32_t* lists[3] = {h->list_def[in][0], h->list_def[in][1], h->list_def[in][2]};
    if ((rc = launch_a(lists, cnt + 3 + 3 * in, out))) return rc;
    in = out;
    ++passes;
  }
  h->stats[0] = passes;
  h->stats[1] = deferred_total;
  h->stats[4] = h->host_counters[9];
  if (h->timing) CB_CUDA(h, cudaEventRecord(h->ev[2], s));
  // phase B
  k_phase_b_warp<<<wgrid, 256, 0, s>>>(c, h->list[0], cnt + 0);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_b_block<kMedThreads><<<mgrid, kMedThreads, 0, s>>>(c, h->list[1], cnt + 1);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_b_block<kBigThreads><<<static_cast<unsigned>(h->num_sms * 2), kBigThreads, 0, s>>>(c, h->list[2], cnt + 2);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  if (h->timing) {
    CB_CUDA(h, cudaEventRecord(h->ev[3], s));
    CB_CUDA(h, cudaEventSynchronize(h->ev[3]));
    float a = 0, b = 0, d = 0, tot = 0;
    CB_CUDA(h, cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    CB_CUDA(h, cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
    CB_CUDA(h, cudaEventElapsedTime(&d, h->ev[2], h->ev[3]));
    CB_CUDA(h, cudaEventElapsedTime(&tot, h->ev[0], h->ev[3]));
    h->phase_ms[0] += a;
    h->phase_ms[1] += b;
    h->phase_ms[2] += d;
    h->phase_ms[3] += tot;
  }
  h->cur = nxt;
  h->g += 1;
  return CB_OK;
}

}  // namespace cb
