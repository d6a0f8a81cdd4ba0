// One global trade (Def. "Undirected Global Trade", Section 3.3) on the GPU.
//
// Layout: during super step g the graph is stored in position space -- row p
// holds the node at position p of the step's permutation, and every entry is
// the neighbour's position, rows ascending.  Trade t owns rows 2t (u_t) and
// 2t+1 (v_t); the neighbour at position y belongs to trade y>>1.
//
// Edges joining trades s and t form a "block" (at most four edges).  A later
// trade t only depends on an earlier trade s when the block has at least two
// edges and one of t's nodes is adjacent to exactly one of s's nodes: only
// then can s's choice change which of t's neighbours are common.  Everywhere
// else the trades are independent because each shuffle key belongs to an edge
// (its endpoints' positions at the start of the step), not to a node.  So the
// step runs in two phases:
//
//  A. Every trade computes D = (A_u u A_v) \ (A_u n A_v) \ {u, v}
//     (Def. "Simple Undirected Trade"), keys its elements, and publishes the
//     threshold (key, lo, hi) of its |A_{u-v}|-th smallest element: u keeps
//     exactly the elements at or below it (Fig. 2: u receives the first
//     |A_{u-v}| elements of sigma(D)).  A trade with an unresolved dependency
//     is deferred to a later pass.  Per entry it stores whether its own trade
//     moves the edge and whether the far trade will consider it.
//  B. Every trade rebuilds its two rows for step g+1: each entry goes to u or
//     v by its own trade's decision, its far end is resolved against the far
//     trade's threshold, positions are mapped to step g+1 and the rows sorted.
//
// Trades of at most `warp_max` entries run on one warp; larger ones on a CTA
// with shared memory, or a global-memory slice above `smem_max` entries.
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

struct StepCtx {
  int64_t n, T;
  uint64_t seed;
  uint32_t g, stamp;
  const int64_t* rp;
  const int32_t* col;
  uint8_t* stash;
  uint64_t* thr_key;
  uint64_t* thr_tb;
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

// Does trade s (owner of positions 2s, 2s+1) send the edge (x, y) to its node
// 2s?  (lo, hi) = step-start positions of the edge.
__device__ __forceinline__ bool far_keeps_low(const StepCtx& c, int64_t s, uint32_t lo, uint32_t hi) {
  const uint64_t k = edge_key(c.seed, lo, hi, c.g, (lo >> 1) == static_cast<uint32_t>(s));
  return at_or_below(k, tie_break(lo, hi), __ldcg(c.thr_key + s), __ldcg(c.thr_tb + s));
}

// Index of value v in sorted row[0..len), or -1.
__device__ __forceinline__ int find_in(const int32_t* row, int len, int32_t v) {
  const int k = lower_bound(row, len, v);
  return (k < len && row[k] == v) ? k : -1;
}

// Workspace of phase A for a trade of L entries.
struct WsA {
  uint64_t* key;
  int32_t* y;
  uint32_t* hist;
  uint8_t* meta;
};

__host__ __device__ inline size_t ws_a_bytes(int L) {
  return ((size_t(L) * 8 + 15) & ~size_t(15)) + ((size_t(L) * 4 + 15) & ~size_t(15)) + 1024 + size_t(L) + 64;
}
__device__ inline WsA carve_a(void* base, int L) {
  char* p = static_cast<char*>(base);
  WsA w;
  w.key = reinterpret_cast<uint64_t*>(p); p += (size_t(L) * 8 + 15) & ~size_t(15);
  w.y = reinterpret_cast<int32_t*>(p); p += (size_t(L) * 4 + 15) & ~size_t(15);
  w.hist = reinterpret_cast<uint32_t*>(p); p += 1024;
  w.meta = reinterpret_cast<uint8_t*>(p);
  return w;
}

// k-th smallest (1-based) of (key, tie-break) over D's elements: MSB-first
// radix select on the 64-bit keys, exact ties broken by (lo, hi).
template <class Team>
__device__ void select_kth(Team& tm, const WsA& w, int L, int64_t t, int k, SelOut* out) {
  uint64_t prefix = 0;
  int shift = 56, kk = k, cnt = 0;
  constexpr int BPM = (256 + Team::N - 1) / Team::N;
  for (;;) {
    for (int b = tm.rank; b < 256; b += Team::N) w.hist[b] = 0;
    tm.sync();
    const uint64_t him = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    for (int i = tm.rank; i < L; i += Team::N)
      if ((w.meta[i] & kInD) && ((w.key[i] & him) == (prefix & him)))
        atomicAdd(&w.hist[(w.key[i] >> shift) & 255u], 1u);
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
        const int hcount = static_cast<int>(w.hist[b]);
        if (below < kk && kk <= below + hcount) {
          out->bin = b;
          out->below = below;
          out->cnt = hcount;
        }
        below += hcount;
      }
    }
    tm.sync();
    kk -= out->below;
    cnt = out->cnt;
    prefix |= static_cast<uint64_t>(out->bin) << shift;
    tm.sync();
    if (cnt == 1 || shift == 0) break;
    shift -= 8;
  }
  const uint64_t msk = ~0ull << shift;
  const uint32_t base = static_cast<uint32_t>(2 * t);
  if (cnt == 1) {
    for (int i = tm.rank; i < L; i += Team::N) {
      if ((w.meta[i] & kInD) && (w.key[i] & msk) == prefix) {
        const uint32_t x = base + (w.meta[i] & kR), y = static_cast<uint32_t>(w.y[i]);
        out->key = w.key[i];
        out->tb = tie_break(min(x, y), max(x, y));
      }
    }
  } else {  // several elements share the full 64-bit key: order them by (lo, hi)
    for (int i = tm.rank; i < L; i += Team::N) {
      if (!(w.meta[i] & kInD) || w.key[i] != prefix) continue;
      const uint32_t xi = base + (w.meta[i] & kR), yi = static_cast<uint32_t>(w.y[i]);
      const uint64_t tbi = tie_break(min(xi, yi), max(xi, yi));
      int r = 0;
      for (int j = 0; j < L; ++j) {
        if (!(w.meta[j] & kInD) || w.key[j] != prefix) continue;
        const uint32_t xj = base + (w.meta[j] & kR), yj = static_cast<uint32_t>(w.y[j]);
        r += tie_break(min(xj, yj), max(xj, yj)) < tbi;
      }
      if (r == kk - 1) {
        out->key = prefix;
        out->tb = tbi;
      }
    }
  }
  tm.sync();
}

// Phase A for trade t.
template <class Team>
__device__ void phase_a(Team& tm, const StepCtx& c, int64_t t, const WsA& w, SelOut* sel) {
  const TradeRows tr = trade_rows(c, t);
  const int du = tr.du, dv = tr.dv, L = du + dv;
  for (int i = tm.rank; i < L; i += Team::N) w.y[i] = __ldcg(c.col + tr.b0 + i);
  tm.sync();
  const int32_t* ru = w.y;
  const int32_t* rv = w.y + du;
  const int64_t t2 = 2 * t;
  bool defer = false;
  int cnt_d = 0, cnt_a = 0;
  for (int i = tm.rank; i < L; i += Team::N) {
    const int r = i >= du;
    const int32_t yy = w.y[i];
    const int64_t s = yy >> 1;
    if (s == t) {
      w.meta[i] = static_cast<uint8_t>(r | kUV);
      continue;
    }
    // initial block matrix between trade t and trade s
    const int32_t e0 = static_cast<int32_t>(2 * s);
    const int li = r ? i - du : i;
    const int32_t* own = r ? rv : ru;
    const int olen = r ? dv : du;
    int own0, own1;
    if (yy & 1) { own1 = 1; own0 = (li > 0 && own[li - 1] == e0) ? 1 : 0; }
    else { own0 = 1; own1 = (li + 1 < olen && own[li + 1] == e0 + 1) ? 1 : 0; }
    const int32_t* oth = r ? ru : rv;
    const int othlen = r ? du : dv;
    const int k0 = lower_bound(oth, othlen, e0);
    const int oth0 = (k0 < othlen && oth[k0] == e0) ? 1 : 0;
    const int k1 = k0 + oth0;
    const int oth1 = (k1 < othlen && oth[k1] == e0 + 1) ? 1 : 0;
    const int u0 = r ? oth0 : own0, u1 = r ? oth1 : own1;
    const int v0 = r ? own0 : oth0, v1 = r ? own1 : oth1;
    const int cu = u0 + u1, cv = v0 + v1;
    uint8_t m = static_cast<uint8_t>(r | (u0 << 4) | (u1 << 5) | (v0 << 6) | (v1 << 7));
    int col_now = yy & 1;                              // s-node of this edge when t acts
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
      for (int rho = 0; rho < 2; ++rho)
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
    if (!other && !tr.single) {
      m |= kInD;
      const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(yy);
      const uint32_t lo = min(x, y), hi = max(x, y);
      w.key[i] = edge_key(c.seed, lo, hi, c.g, (lo >> 1) == static_cast<uint32_t>(t));
      ++cnt_d;
      cnt_a += (r == 0);
    }
    w.meta[i] = m;
  }
  if (tm.any(defer)) {
    if (tm.rank == 0) c.def_out[atomicAdd(c.def_count, 1)] = static_cast<int32_t>(t);
    tm.sync();
    return;
  }
  const int nd = static_cast<int>(tm.sum(cnt_d));
  const int a = static_cast<int>(tm.sum(cnt_a));
  uint64_t tk = 0, tt = 0;
  if (!tr.single && a > 0) {
    select_kth(tm, w, L, t, a, sel);
    tk = sel->key;
    tt = sel->tb;
  }
  (void)nd;
  // own decisions
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    if (!(m & kInD)) continue;
    const int r = m & kR;
    const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(w.y[i]);
    const int newr = at_or_below(w.key[i], tie_break(min(x, y), max(x, y)), tk, tt) ? 0 : 1;
    if (newr != r) w.meta[i] = m | kFlip;
  }
  tm.sync();
  // will the far trade consider this edge?
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
          const int myrow = r ^ f;
          int same = 0;
          const int bits[4] = {u0, u1, v0, v1};
          for (int q = 0; q < 4; ++q) {
            if (!bits[q]) continue;
            const int rho = q >> 1, gam = q & 1;
            const int idx = rho ? du + find_in(rv, dv, e0 + gam) : find_in(ru, du, e0 + gam);
            const int fj = (w.meta[idx] & kFlip) ? 1 : 0;
            same += ((rho ^ fj) == myrow);
          }
          in_far = (same == 1);
        }
      }
    }
    c.stash[tr.b0 + i] = static_cast<uint8_t>(f | (in_far << 1));
  }
  if (tm.rank == 0 && !tr.single) {
    c.thr_key[t] = tk;
    c.thr_tb[t] = tt;
    __threadfence();
    st_release(c.done + t, c.stamp);
  }
  tm.sync();
}

// Phase B for trade t: rebuild its two rows in step g+1's layout.
template <class Team>
__device__ void phase_b(Team& tm, const StepCtx& c, int64_t t, uint64_t* wbuf) {
  const TradeRows tr = trade_rows(c, t);
  const int du = tr.du, dv = tr.dv, L = du + dv;
  const int P = next_pow2(L);
  const int64_t t2 = 2 * t;
  for (int i = tm.rank; i < P; i += Team::N) {
    uint64_t v = ~0ull;
    if (i < L) {
      const int r = i >= du;
      const int32_t yy = __ldcg(c.col + tr.b0 + i);
      const uint8_t st = c.stash[tr.b0 + i];
      const int r2 = r ^ (st & 1);
      int32_t y2 = yy;
      if (st & 2) {
        const int64_t s = yy >> 1;
        const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(yy);
        y2 = static_cast<int32_t>(2 * s) + (far_keeps_low(c, s, min(x, y), max(x, y)) ? 0 : 1);
      }
      v = (static_cast<uint64_t>(r2) << 32) | static_cast<uint32_t>(c.M[y2]);
    }
    wbuf[i] = v;
  }
  tm.sync();
  team_bitonic_sort(tm, wbuf, P);
  const int32_t pu = c.M[t2];
  const int64_t ou = c.rp_next[pu];
  if (c.rp_next[pu + 1] - ou != du) {
    if (tm.rank == 0) latch(c.err, kErrRowLength);
    tm.sync();
    return;
  }
  int64_t ov = 0;
  if (dv > 0) {
    const int32_t pv = c.M[t2 + 1];
    ov = c.rp_next[pv];
    if (c.rp_next[pv + 1] - ov != dv) {
      if (tm.rank == 0) latch(c.err, kErrRowLength);
      tm.sync();
      return;
    }
  }
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint64_t v = wbuf[i];
    const int side = static_cast<int>(v >> 32);
    if (side != (i >= du)) latch(c.err, kErrRowSide);
    if (i < du) c.col_next[ou + i] = static_cast<int32_t>(static_cast<uint32_t>(v));
    else c.col_next[ov + (i - du)] = static_cast<int32_t>(static_cast<uint32_t>(v));
  }
  tm.sync();
}

// ---------------------------------------------------------------- kernels

__global__ void k_classify(StepCtx c, int64_t ntasks, int warp_max, int32_t* __restrict__ lw,
                           int32_t* __restrict__ lb, int32_t* __restrict__ counters) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < ntasks; t += int64_t(gridDim.x) * blockDim.x) {
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    if (L <= warp_max) lw[atomicAdd(&counters[0], 1)] = static_cast<int32_t>(t);
    else lb[atomicAdd(&counters[1], 1)] = static_cast<int32_t>(t);
  }
}

struct WarpWsA {
  uint64_t key[kWarpCapMax];
  int32_t y[kWarpCapMax];
  uint32_t hist[256];
  uint8_t meta[kWarpCapMax];
  SelOut sel;
};

__global__ void __launch_bounds__(256) k_phase_a_warp(StepCtx c, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ count) {
  __shared__ WarpWsA ws[kWarpsPerCta];
  WarpTeam tm;
  const int wid = threadIdx.x >> 5;
  WsA w{ws[wid].key, ws[wid].y, ws[wid].hist, ws[wid].meta};
  const int64_t len = *count;
  for (int64_t q = blockIdx.x * int64_t(kWarpsPerCta) + wid; q < len; q += int64_t(gridDim.x) * kWarpsPerCta)
    phase_a(tm, c, list[q], w, &ws[wid].sel);
}

__global__ void __launch_bounds__(kBlockThreads) k_phase_a_block(StepCtx c, const int32_t* __restrict__ list,
                                                                 const int32_t* __restrict__ count, int smem_max,
                                                                 char* gws, size_t slice) {
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[kBlockThreads / 32 + 2];
  __shared__ SelOut sel;
  BlockTeam<kBlockThreads> tm(red);
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
  __shared__ uint64_t ws[kWarpsPerCta][kWarpCapMax];
  WarpTeam tm;
  const int wid = threadIdx.x >> 5;
  const int64_t len = *count;
  for (int64_t q = blockIdx.x * int64_t(kWarpsPerCta) + wid; q < len; q += int64_t(gridDim.x) * kWarpsPerCta)
    phase_b(tm, c, list[q], ws[wid]);
}

__global__ void __launch_bounds__(kBlockThreads) k_phase_b_block(StepCtx c, const int32_t* __restrict__ list,
                                                                 const int32_t* __restrict__ count, int smem_max,
                                                                 char* gws, size_t slice) {
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[kBlockThreads / 32 + 2];
  BlockTeam<kBlockThreads> tm(red);
  const int64_t len = *count;
  for (int64_t q = blockIdx.x; q < len; q += gridDim.x) {
    const int64_t t = list[q];
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    char* base = (L > smem_max) ? gws + slice * blockIdx.x : sbuf;
    phase_b(tm, c, t, reinterpret_cast<uint64_t*>(base));
  }
}

size_t block_smem_bytes(int smem_max) {
  const size_t a = ws_a_bytes(smem_max);
  const size_t b = static_cast<size_t>(next_pow2_host(smem_max)) * 8;
  return std::max(a, b);
}

}  // namespace

size_t trade_ws_slice_bytes(int64_t max_trade) {
  const size_t a = ws_a_bytes(static_cast<int>(max_trade));
  const size_t b = static_cast<size_t>(next_pow2_host(max_trade)) * 8;
  return (std::max(a, b) + 255) & ~size_t(255);
}

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
  c.done = h->done;
  c.err = h->err;
  c.M = h->M;
  c.rp_next = h->rp[nxt];
  c.col_next = h->col[nxt];
  c.gws_count = h->counters + 6;
  int32_t* cnt = h->counters;
  CB_CUDA(h, cudaMemsetAsync(cnt, 0, 8 * sizeof(int32_t), s));
  const int64_t ntasks = h->ntasks;
  if (ntasks == 0) {
    h->cur = nxt;
    h->g += 1;
    return CB_OK;
  }
  const int warp_max = std::min(h->warp_max, kWarpCapMax);
  {
    const int64_t want = (ntasks + 255) / 256;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, h->num_sms * 8)));
    k_classify<<<grid, 256, 0, s>>>(c, ntasks, warp_max, h->list_warp, h->list_block, cnt);
    CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  }
  const unsigned wgrid = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>((ntasks + kWarpsPerCta - 1) / kWarpsPerCta, h->num_sms * 8)));
  const size_t bsmem = block_smem_bytes(h->smem_max);
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(bsmem)));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_b_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(bsmem)));
  const unsigned bgrid = static_cast<unsigned>(std::max(1, h->ws_ctas));
  char* gws = static_cast<char*>(h->ws_global);

  // phase A, first pass over all trades
  c.def_out = h->list_def[0];
  c.def_count = cnt + 2;
  k_phase_a_warp<<<wgrid, 256, 0, s>>>(c, h->list_warp, cnt + 0);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_a_block<<<bgrid, kBlockThreads, bsmem, s>>>(c, h->list_block, cnt + 1, h->smem_max, gws, h->ws_slice);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  // further passes over deferred trades until none is left
  int64_t passes = 1, deferred_total = 0;
  int in = 0;
  for (;;) {
    CB_CUDA(h, cudaMemcpyAsync(h->host_counters, cnt, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CB_CUDA(h, cudaStreamSynchronize(s));
    const int32_t ndef = h->host_counters[2 + in];
    if (passes == 1) {
      h->stats[2] = h->host_counters[0];
      h->stats[3] = h->host_counters[1];
    }
    if (ndef == 0) break;
    deferred_total += ndef;
    if (passes > 100000) return fail(h, CB_ECHECK, "dependency resolution did not converge");
    const int out = 1 - in;
    CB_CUDA(h, cudaMemsetAsync(cnt + 2 + out, 0, sizeof(int32_t), s));
    c.def_out = h->list_def[out];
    c.def_count = cnt + 2 + out;
    k_phase_a_block<<<bgrid, kBlockThreads, bsmem, s>>>(c, h->list_def[in], cnt + 2 + in, h->smem_max, gws,
                                                        h->ws_slice);
    CB_CUDA(h, cudaGetLastError());
  ++h->launches;
    in = out;
    ++passes;
  }
  h->stats[0] = passes;
  h->stats[1] = deferred_total;
  h->stats[4] = h->host_counters[6];
  if (h->timing) CB_CUDA(h, cudaEventRecord(h->ev[2], s));
  // phase B
  k_phase_b_warp<<<wgrid, 256, 0, s>>>(c, h->list_warp, cnt + 0);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_b_block<<<bgrid, kBlockThreads, bsmem, s>>>(c, h->list_block, cnt + 1, h->smem_max, gws, h->ws_slice);
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
