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
//     published yet is marked deferred; one more pass runs the deferred
//     trades in index order (see k_phase_a_inorder).  Per entry it stores one
//     byte: whether its own trade moves the edge, whether the far trade will
//     consider the edge, and the top six bits of the far trade's key for it.
//  B. Every trade writes its two rows for step g+1: each entry goes to u or v
//     by its own trade's bit; its far end is resolved against the far trade's
//     threshold (six-bit prefix first, the full key only on a prefix tie), and
//     positions are mapped to step g+1.  One flat pass over all entries.
//
// Phase A by trade size: trades of at most `tile_max` entries run on the tile
// path (a CTA takes a run of consecutive small trades, about 1024 entries,
// one thread per entry); trades up to `block_max` entries run one per
// 256-thread CTA, larger ones one per 1024-thread CTA with up to `smem_max`
// entries in shared memory (a global-memory slice above that).
#include <algorithm>

#include "cb_internal.cuh"
#include "philox.cuh"
#include "team.cuh"

namespace cb {
namespace {

constexpr uint32_t kDeferred = 2;              // done[t]: deferred by the first pass
constexpr uint32_t kWaitLimit = 1u << 24;      // polls of a dependency before giving up (about 2 s)

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
constexpr int kTileThreads = 256;
constexpr int kTileCap = 1024;                       // weight units per tile (weight = max(L, 4))
constexpr int kTileTrades = kTileCap / 4;            // so at most 256 trades per tile
constexpr int kTileSlots = kTileCap + kTileMaxCap;   // a trade may start just before the cap
constexpr int kNoOwner = 0xFFFF;
constexpr int kTileHashLg = 11;
constexpr int kTileHash = 1 << kTileHashLg;          // > 1.7 x the slots of a tile

struct StepCtx {
  int64_t n, T;
  uint32_t stamp;
  const Seg* segs;          // per graph: seed, step, first position
  const int32_t* seg_of;    // graph of each position (null: one graph)
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
  unsigned long long* def_count;   // trades deferred by the first pass
  uint32_t wait;                   // 0: defer a trade whose dependency is unpublished; 1: wait for it
  unsigned long long* gws_count;
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

// ------------------------------------------------- bulk copies (TMA engine)
//
// A trade's entries are staged into shared memory by one cp.async.bulk copy
// that completes on an mbarrier.  The copy moves whole 16-byte units, so it
// starts at the entry rounded down to a multiple of 4 and covers a multiple
// of 4 entries; the adjacency buffers carry 16 spare entries at their end, so
// the copy never leaves its allocation.

constexpr uint32_t kTmaWaitLimit = 1u << 23;   // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of m (non-blocking polls with a short
// sleep, about a second at most); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  for (uint32_t it = 0; it < kTmaWaitLimit; ++it) {
    if (mbar_test_wait(m, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// Entries [b0, b0 + L) of col staged at buf + stage_off(b0).
__device__ __forceinline__ int stage_off(int64_t b0) { return static_cast<int>(b0 & 3); }
__device__ __forceinline__ void stage_issue(const int32_t* col, int64_t b0, int L, int32_t* buf, uint64_t* m) {
  const int64_t a0 = b0 & ~int64_t(3);
  const uint32_t bytes = static_cast<uint32_t>(((b0 + L - a0) + 3) & ~int64_t(3)) * 4u;
  fence_proxy_async();   // earlier generic reads of buf come before the copy's writes
  mbar_expect_tx(m, bytes);
  bulk_g2s(buf, col + a0, bytes, m);
}

__device__ __forceinline__ uint64_t tie_break(uint32_t lo, uint32_t hi) {
  return (static_cast<uint64_t>(lo) << 32) | hi;
}
// (key, tb) <= (tk, tt), lexicographic
__device__ __forceinline__ bool at_or_below(uint64_t key, uint64_t tb, uint64_t tk, uint64_t tt) {
  return key < tk || (key == tk && tb <= tt);
}

// Key parameters of a trade's graph: its seed, its step and its first
// position (keys count positions from the start of the graph).  Both ends of
// an edge are in the same graph.
struct KeyCtx {
  uint64_t seed;
  uint32_t g, off;
};
__device__ __forceinline__ KeyCtx key_ctx(const StepCtx& c, int64_t t) {
  const Seg* S = c.segs + (c.seg_of ? __ldg(c.seg_of + 2 * t) : 0);
  return {__ldg(&S->seed), __ldg(&S->g), static_cast<uint32_t>(__ldg(&S->off))};
}

// Both trades' keys of the edge whose step-start positions are lo < hi.
struct EdgeKeys {
  uint64_t lo_side, hi_side;
};
__device__ __forceinline__ EdgeKeys edge_keys(const KeyCtx& kc, uint32_t lo, uint32_t hi) {
  const Philox4 r = philox4x32_10(lo - kc.off, hi - kc.off, kc.g, 1u, kc.seed);
  return {(static_cast<uint64_t>(r.w0) << 32) | r.w1, (static_cast<uint64_t>(r.w2) << 32) | r.w3};
}
__device__ __forceinline__ uint64_t side_key(const KeyCtx& kc, uint32_t lo, uint32_t hi, bool lo_side) {
  return edge_key(kc.seed, lo - kc.off, hi - kc.off, kc.g, lo_side);
}

// Does trade s send the edge (lo, hi) to its node at position 2s?  Full test.
__device__ __forceinline__ bool far_keeps_low(const StepCtx& c, const KeyCtx& kc, int64_t s, uint32_t lo,
                                              uint32_t hi) {
  const uint64_t k = side_key(kc, lo, hi, (lo >> 1) == static_cast<uint32_t>(s));
  return at_or_below(k, tie_break(lo, hi), __ldcg(c.thr_key + s), __ldcg(c.thr_tb + s));
}

// ------------------------------------------------------------ hash table
//
// One slot per far trade s of the current trade: key s + 1 (0 = empty) and a
// flag byte: bit (2 rho + gamma) = the trade's node at row rho (0: u, 1: v) is
// adjacent to s's node at position 2s + gamma (the 2x2 block matrix), bit
// (4 + 2 rho + gamma) = that entry is moved by the trade (its flip).

__device__ __forceinline__ uint32_t hslot(uint32_t s, int lgH) { return (s * 0x9E3779B1u) >> (32 - lgH); }

__device__ __forceinline__ void flag_or(uint8_t* fl, int p, uint32_t bits) {
  atomicOr(reinterpret_cast<unsigned int*>(fl + (p & ~3)), bits << (8 * (p & 3)));
}

// Sets `bit` in the slot of far trade s (creating it); returns the slot.
__device__ __forceinline__ int h_insert(uint32_t* hk, uint8_t* fl, int lgH, uint32_t s, uint32_t bit) {
  const uint32_t key = s + 1u;
  const uint32_t mask = (1u << lgH) - 1u;
  uint32_t p = hslot(s, lgH);
  for (;;) {
    uint32_t cur = hk[p];
    if (cur == 0) {
      cur = atomicCAS(&hk[p], 0u, key);
      if (cur == 0) cur = key;
    }
    if (cur == key) {
      flag_or(fl, static_cast<int>(p), bit);
      return static_cast<int>(p);
    }
    p = (p + 1) & mask;
  }
}

// ---------------------------------------------------------- workspace

constexpr int kSelBits = 10;              // first radix digit: top 10 bits of the key
constexpr int kSelBins = 1 << kSelBits;

// meta bits per entry (team paths add the neighbour's column bit)
constexpr uint8_t kCol = 16;    // neighbour sits at the odd position 2s+1

constexpr int kCand = 32;       // candidates sharing the threshold's bin, ranked by full key

struct WsA {
  uint64_t* ck;               // kCand candidate keys
  uint64_t* ctb;              // their tie-breaks
  int32_t* cidx;              // their entry indices
  int32_t* ncand;
  int32_t* slot;              // hash slot of the entry's far trade (-1: the edge {u,v})
  uint16_t* top;              // top 16 bits of the own key
  uint8_t* meta;
  uint8_t* far;               // top 6 bits of the far trade's key
  uint32_t* hkey;             // 2^lgH slot keys
  uint8_t* hflag;             // 2^lgH slot flag bytes
  uint32_t* hist;             // kSelBins bins
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
  const size_t H = size_t(1) << hash_lg(L);
  return H * 4 + ((H + 15) & ~size_t(15)) + kSelBins * 4 + kCand * 20 + 16 + L16 * 4 + L16 * 2 + L16 + L16 + 64;
}
// Dynamic shared memory of k_phase_a_block: workspace for `cap` entries, then
// the staging buffer of a trade's entries.
inline size_t block_smem_bytes(int cap) {
  return ((ws_a_bytes(cap) + 127) & ~size_t(127)) + (static_cast<size_t>(cap) + 8) * 4;
}

__device__ inline WsA carve_a(void* base, int L) {
  const size_t L16 = (static_cast<size_t>(L) + 15) & ~size_t(15);
  char* p = static_cast<char*>(base);
  WsA w;
  w.lgH = hash_lg(L);
  const size_t H = size_t(1) << w.lgH;
  w.hkey = reinterpret_cast<uint32_t*>(p); p += H * 4;
  w.hflag = reinterpret_cast<uint8_t*>(p); p += (H + 15) & ~size_t(15);
  w.hist = reinterpret_cast<uint32_t*>(p); p += kSelBins * 4;
  w.ck = reinterpret_cast<uint64_t*>(p); p += kCand * 8;
  w.ctb = reinterpret_cast<uint64_t*>(p); p += kCand * 8;
  w.cidx = reinterpret_cast<int32_t*>(p); p += kCand * 4;
  w.ncand = reinterpret_cast<int32_t*>(p); p += 16;
  w.slot = reinterpret_cast<int32_t*>(p); p += L16 * 4;
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
__device__ __forceinline__ uint64_t own_key(const KeyCtx& kc, int64_t t, uint32_t lo, uint32_t hi) {
  return side_key(kc, lo, hi, (lo >> 1) == static_cast<uint32_t>(t));
}
// The neighbour position of a team-path entry (its far trade from the hash).
__device__ __forceinline__ int32_t entry_y(const WsA& w, int64_t t2, int i) {
  const uint8_t m = w.meta[i];
  if (m & kUV) return static_cast<int32_t>(t2 + 1 - (m & kR));
  const uint32_t s = w.hkey[w.slot[i]] - 1u;
  return static_cast<int32_t>(2 * s + ((m & kCol) ? 1 : 0));
}

// One radix digit of the 16-bit key prefixes: histogram of bits
// [shift, shift + bits) over the elements of D whose bits above equal `pre`
// (all of D when shift + bits == 16), then the bin holding the kk-th element.
template <class Team>
__device__ void radix_digit(Team& tm, const WsA& w, int L, int shift, int bits, uint32_t pre, int kk, SelOut* out) {
  const int nb = 1 << bits;
  const int bpm = (nb + Team::N - 1) / Team::N;
  for (int b = tm.rank; b < nb; b += Team::N) w.hist[b] = 0;
  tm.sync();
  for (int i = tm.rank; i < L; i += Team::N) {
    if (!(w.meta[i] & kInD)) continue;
    const uint32_t tp = w.top[i];
    if (shift + bits == 16 || (tp >> (shift + bits)) == pre) atomicAdd(&w.hist[(tp >> shift) & (nb - 1)], 1u);
  }
  tm.sync();
  const int b0 = tm.rank * bpm;
  int local = 0;
  for (int j = 0; j < bpm; ++j)
    if (b0 + j < nb) local += static_cast<int>(w.hist[b0 + j]);
  int below = static_cast<int>(tm.exscan(local));
  for (int j = 0; j < bpm; ++j) {
    const int b = b0 + j;
    if (b < nb) {
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

// k-th smallest (1-based) (key, lo, hi) over D, the general procedure (used
// when more than kCand elements share the threshold's bin): one 10-bit radix digit on the
// stored 16-bit key prefixes (keys are uniform, so the chosen bin holds about
// |D|/1024 elements), a 6-bit digit only if that bin is crowded, then the
// full keys of the few remaining candidates.
template <class Team>
__device__ void select_kth(Team& tm, const KeyCtx& kc, const WsA& w, int L, int64_t t, int k, SelOut* out) {
  const int64_t t2 = 2 * t;
  radix_digit(tm, w, L, 16 - kSelBits, kSelBits, 0, k, out);
  uint32_t prefix = static_cast<uint32_t>(out->bin);   // of the top `plen` bits
  int plen = kSelBits;
  int kk = k - out->below;
  int cnt = out->cnt;
  tm.sync();
  if (cnt > kCand) {
    radix_digit(tm, w, L, 0, 16 - kSelBits, prefix, kk, out);
    prefix = (prefix << (16 - kSelBits)) | static_cast<uint32_t>(out->bin);
    plen = 16;
    kk -= out->below;
    cnt = out->cnt;
    tm.sync();
  }
  uint64_t* ck = reinterpret_cast<uint64_t*>(w.hist);
  uint64_t* ctb = ck + kCand;
  int* ncand = reinterpret_cast<int*>(ctb + kCand);
  if (cnt > 1 && cnt <= kCand) {
    if (tm.rank == 0) *ncand = 0;
    tm.sync();
  }
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    if (!(m & kInD)) continue;
    if ((static_cast<uint32_t>(w.top[i]) >> (16 - plen)) != prefix) continue;
    const int32_t y = entry_y(w, t2, i);
    const uint32_t lo = lo_of(t2, m, y), hi = hi_of(t2, m, y);
    const uint64_t ki = own_key(kc, t, lo, hi), tbi = tie_break(lo, hi);
    if (cnt == 1) {            // the only element with this prefix
      out->key = ki;
      out->tb = tbi;
    } else if (cnt <= kCand) {
      const int q = atomicAdd(ncand, 1);
      ck[q] = ki;
      ctb[q] = tbi;
    } else {                   // many equal 16-bit prefixes: rank against every other candidate
      int r = 0;
      for (int j = 0; j < L; ++j) {
        const uint8_t mj = w.meta[j];
        if (j == i || !(mj & kInD)) continue;
        if ((static_cast<uint32_t>(w.top[j]) >> (16 - plen)) != prefix) continue;
        const int32_t yj = entry_y(w, t2, j);
        const uint32_t loj = lo_of(t2, mj, yj), hij = hi_of(t2, mj, yj);
        const uint64_t kj = own_key(kc, t, loj, hij);
        r += (kj < ki || (kj == ki && tie_break(loj, hij) < tbi));
      }
      if (r == kk - 1) {
        out->key = ki;
        out->tb = tbi;
      }
    }
  }
  tm.sync();
  if (cnt > 1 && cnt <= kCand) {
    for (int q = tm.rank; q < cnt; q += Team::N) {
      int r = 0;
      for (int j = 0; j < cnt; ++j) r += (ck[j] < ck[q] || (ck[j] == ck[q] && ctb[j] < ctb[q]));
      if (r == kk - 1) {
        out->key = ck[q];
        out->tb = ctb[q];
      }
    }
    tm.sync();
  }
}

// Phase A for trade t.
// The next trade's bulk copy, issued by member 0 as soon as the current trade
// has read its staged entries (the same buffer is reused).
struct StageNext {
  bool issue;
  int64_t b0;
  int L;
  int32_t* buf;
  uint64_t* mbar;
};

template <class Team>
__device__ void phase_a(Team& tm, const StepCtx& c, int64_t t, const WsA& w, SelOut* sel,
                        const int32_t* ystage = nullptr, StageNext sn = StageNext{false, 0, 0, nullptr, nullptr}) {
  const TradeRows tr = trade_rows(c, t);
  const KeyCtx kc = key_ctx(c, t);
  const int du = tr.du, dv = tr.dv, L = du + dv;
  const int H = 1 << w.lgH;
  const int64_t t2 = 2 * t;
  for (int i = tm.rank; i < H; i += Team::N) w.hkey[i] = 0u;
  for (int i = tm.rank; i < ((H + 15) & ~15) / 4; i += Team::N) reinterpret_cast<uint32_t*>(w.hflag)[i] = 0u;
  for (int i = tm.rank; i < kSelBins; i += Team::N) w.hist[i] = 0;
  if (tm.rank == 0) *w.ncand = 0;
  tm.sync();
  // entries into the hash: presence bit (row, column) in the far trade's slot
  for (int i = tm.rank; i < L; i += Team::N) {
    const int r = i >= du;
    const int32_t yy = ystage ? ystage[i] : __ldcg(c.col + tr.b0 + i);
    const int64_t s = yy >> 1;
    uint8_t m = static_cast<uint8_t>(r | ((yy & 1) ? kCol : 0));
    if (s == t) {
      m |= kUV;
      w.slot[i] = -1;
    } else {
      w.slot[i] = h_insert(w.hkey, w.hflag, w.lgH, static_cast<uint32_t>(s), 1u << (2 * r + (yy & 1)));
    }
    w.meta[i] = m;
  }
  tm.sync();
  if (sn.issue && tm.rank == 0) stage_issue(c.col, sn.b0, sn.L, sn.buf, sn.mbar);
  // trade and position indices fit 32 bits (n < 2^31)
  const uint32_t t32 = static_cast<uint32_t>(t), T32 = static_cast<uint32_t>(c.T);
  const uint32_t t2u = 2u * t32;
  bool defer = false, has_dependents = false;
  int cnt_a = 0;
  for (int i = tm.rank; i < L; i += Team::N) {
    uint8_t m = w.meta[i];
    w.far[i] = 0;
    w.top[i] = 0;
    if (m & kUV) continue;
    const int r = m & kR;
    const uint32_t colb = (m & kCol) ? 1u : 0u;
    const int sl = w.slot[i];
    const uint32_t s = w.hkey[sl] - 1u;
    const uint32_t f = w.hflag[sl] & 15u;
    int other = 0;   // the other row is adjacent to this neighbour (a common neighbour)
    if (f & (f - 1u)) {
      // a block of two or more edges: common neighbours and dependencies
      const int u0 = f & 1, u1 = (f >> 1) & 1, v0 = (f >> 2) & 1, v1 = (f >> 3) & 1;
      const int cu = u0 + u1, cv = v0 + v1;
      // a later trade s depends on t when one of its own nodes holds exactly
      // one of the block's edges
      if (!tr.single && s > t32 && s < T32 && (u0 + v0 == 1 || u1 + v1 == 1)) has_dependents = true;
      int col_now = static_cast<int>(colb);          // s-node of this edge when t acts
      other = r ? (col_now ? u1 : u0) : (col_now ? v1 : v0);
      const bool dep = !tr.single && s < t32 && (cu == 1 || cv == 1);
      if (dep) {
        if (ld_acquire(c.done + s) != c.stamp) {
          if (!c.wait) {
            defer = true;
            continue;
          }
          // in-order pass: s is complete or held by a running CTA that claimed it
          // earlier, so the wait ends; the limit turns a broken invariant into an error
          uint32_t polls = 0;
          while (ld_acquire(c.done + s) != c.stamp) {
            if (++polls > kWaitLimit) {
              latch(c.err, kErrResolve);
              break;
            }
            __nanosleep(128);
          }
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
              const uint32_t x = t2u + rho, y = 2u * s + gam;
              g2 = far_keeps_low(c, kc, s, min(x, y), max(x, y)) ? 0 : 1;
            }
            m1[rho][g2] = 1;
            if (rho == r && gam == static_cast<int>(colb)) col_now = g2;
          }
        other = m1[1 - r][col_now];
      }
    }
    // both trades' keys of this edge: own 16-bit prefix, far 6-bit prefix
    const uint32_t x = t2u + r, y = 2u * s + colb;
    const uint32_t lo = min(x, y), hi = max(x, y);
    const EdgeKeys ek = edge_keys(kc, lo, hi);
    const bool lo_mine = (lo >> 1) == t32;
    const uint32_t top = static_cast<uint32_t>((lo_mine ? ek.lo_side : ek.hi_side) >> 48);
    w.top[i] = static_cast<uint16_t>(top);
    w.far[i] = static_cast<uint8_t>((lo_mine ? ek.hi_side : ek.lo_side) >> 58);
    if (!other && !tr.single) {
      m |= kInD;
      cnt_a += (r == 0);
      atomicAdd(&w.hist[top >> (16 - kSelBits)], 1u);
    }
    w.meta[i] = m;
  }
  // one reduction: |A_{u-v}|, any deferral, any later dependent trade
  const int64_t tot = tm.sum(static_cast<int64_t>(cnt_a) | (static_cast<int64_t>(defer) << 32) |
                             (static_cast<int64_t>(has_dependents) << 48));
  if ((tot >> 32) & 0xffff) {
    if (tm.rank == 0) {
      c.done[t] = kDeferred;
      atomicAdd(c.def_count, 1ull);
    }
    return;
  }
  const int a = static_cast<int>(tot & 0xffffffff);
  const bool publish_fence = (tot >> 48) != 0;
  const bool no_thr = tr.single || a == 0;   // u keeps nothing of D
  // the bin of the top kSelBits key bits that holds the a-th smallest element
  int bin = 0, cnt = 0, below = 0;
  if (!no_thr) {
    constexpr int bpm = (kSelBins + Team::N - 1) / Team::N;
    const int b0 = tm.rank * bpm;
    int local = 0;
#pragma unroll
    for (int j = 0; j < bpm; ++j)
      if (b0 + j < kSelBins) local += static_cast<int>(w.hist[b0 + j]);
    int run = static_cast<int>(tm.exscan(local));
#pragma unroll
    for (int j = 0; j < bpm; ++j) {
      const int b = b0 + j;
      if (b < kSelBins) {
        const int hc = static_cast<int>(w.hist[b]);
        if (run < a && a <= run + hc) {
          sel->bin = b;
          sel->below = run;
          sel->cnt = hc;
        }
        run += hc;
      }
    }
    tm.sync();
    bin = sel->bin;
    below = sel->below;
    cnt = sel->cnt;
  }
  uint64_t tk = 0, tt = 0;
  if (cnt <= kCand) {
    // own decisions: an element below the threshold's bin stays with u, above it
    // goes to v; in the bin, full keys decide (the only element: the threshold)
    for (int i = tm.rank; i < L; i += Team::N) {
      const uint8_t m = w.meta[i];
      if (!(m & kInD)) continue;
      const int r = m & kR;
      const int d = static_cast<int>(w.top[i]) >> (16 - kSelBits);
      bool low;
      if (no_thr || d > bin) {
        low = false;
      } else if (d < bin) {
        low = true;
      } else {
        const int32_t y = entry_y(w, t2, i);
        const uint32_t lo = lo_of(t2, m, y), hi = hi_of(t2, m, y);
        const uint64_t ki = own_key(kc, t, lo, hi), tbi = tie_break(lo, hi);
        if (cnt == 1) {
          low = true;
          sel->key = ki;
          sel->tb = tbi;
        } else {
          const int q = atomicAdd(w.ncand, 1);
          w.ck[q] = ki;
          w.ctb[q] = tbi;
          w.cidx[q] = i;
          continue;
        }
      }
      if ((low ? 0 : 1) != r) {
        w.meta[i] = m | kFlip;
        flag_or(w.hflag, w.slot[i], 16u << (2 * r + ((m & kCol) ? 1 : 0)));
      }
    }
    tm.sync();
    if (cnt > 1) {   // rank the elements of the threshold's bin
      const int kk = a - below;
      for (int q = tm.rank; q < cnt; q += Team::N) {
        int rk = 0;
        for (int j = 0; j < cnt; ++j) rk += (w.ck[j] < w.ck[q] || (w.ck[j] == w.ck[q] && w.ctb[j] < w.ctb[q]));
        if (rk == kk - 1) {
          sel->key = w.ck[q];
          sel->tb = w.ctb[q];
        }
        const int i = w.cidx[q];
        const uint8_t m = w.meta[i];
        const int r = m & kR;
        if ((rk < kk ? 0 : 1) != r) {
          w.meta[i] = m | kFlip;
          flag_or(w.hflag, w.slot[i], 16u << (2 * r + ((m & kCol) ? 1 : 0)));
        }
      }
      tm.sync();
    }
    if (!no_thr) {
      tk = sel->key;
      tt = sel->tb;
    }
  } else {
    // crowded bin (|D| in the tens of thousands): the general selection
    select_kth(tm, kc, w, L, t, a, sel);
    tk = sel->key;
    tt = sel->tb;
    const uint32_t tk16 = static_cast<uint32_t>(tk >> 48);
    for (int i = tm.rank; i < L; i += Team::N) {
      const uint8_t m = w.meta[i];
      if (!(m & kInD)) continue;
      const int r = m & kR;
      const uint32_t tp = w.top[i];
      bool low;
      if (tp != tk16) {
        low = tp < tk16;
      } else {
        const int32_t y = entry_y(w, t2, i);
        const uint32_t lo = lo_of(t2, m, y), hi = hi_of(t2, m, y);
        low = at_or_below(own_key(kc, t, lo, hi), tie_break(lo, hi), tk, tt);
      }
      if ((low ? 0 : 1) != r) {
        w.meta[i] = m | kFlip;
        flag_or(w.hflag, w.slot[i], 16u << (2 * r + ((m & kCol) ? 1 : 0)));
      }
    }
    tm.sync();
  }
  // will the far trade consider this edge?  Write the stash byte.
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    const int f = (m & kFlip) ? 1 : 0;
    int in_far = 0;
    if (!(m & kUV)) {
      const int r = m & kR;
      const int sl = w.slot[i];
      const uint32_t s = w.hkey[sl] - 1u;
      const uint32_t fl = w.hflag[sl];
      const int u0 = fl & 1, u1 = (fl >> 1) & 1, v0 = (fl >> 2) & 1, v1 = (fl >> 3) & 1;
      const int cr = r ? (v0 + v1) : (u0 + u1);
      if (tr.single || s < t32) {
        in_far = (cr == 1);                 // trade s acted before t: initial block
      } else if (s < T32) {
        if (u0 + u1 + v0 + v1 == 1) {
          in_far = 1;
        } else {                            // block after t's own decisions: presence bits 0..3, flips 4..7
          const int myrow = r ^ f;
          int same = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (!((fl >> q) & 1)) continue;
            same += (((q >> 1) ^ ((fl >> (4 + q)) & 1)) == myrow);
          }
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

// ---------------------------------------------------------- classification

// Class of each trade (tile / 256 / 1024 threads) and its tile weight.
__global__ void k_class_flags(StepCtx c, int64_t ntasks, int tile_max, int block_max, int32_t* __restrict__ f) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < ntasks; t += int64_t(gridDim.x) * blockDim.x) {
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    const int cls = L <= tile_max ? 0 : (L <= block_max ? 1 : 2);
    f[t] = cls == 0;
    f[ntasks + t] = cls == 1;
    f[2 * ntasks + t] = cls == 2;
    f[3 * ntasks + t] = cls == 0 ? max(L, kTileCap / kTileTrades) : 0;
  }
}

// Stable compaction of each class into index order, plus tile offsets.
__global__ void k_class_scatter(int64_t ntasks, const int32_t* __restrict__ f, const int64_t* __restrict__ sc,
                                int32_t* __restrict__ l0, int32_t* __restrict__ l1, int32_t* __restrict__ l2,
                                int64_t* __restrict__ tile_off) {
  const int64_t n1 = ntasks + 1;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < ntasks; t += int64_t(gridDim.x) * blockDim.x) {
    if (f[t]) {
      const int64_t k = sc[t];
      l0[k] = static_cast<int32_t>(t);
      tile_off[k] = sc[3 * n1 + t];
    } else if (f[ntasks + t]) {
      l1[sc[n1 + t]] = static_cast<int32_t>(t);
    } else {
      l2[sc[2 * n1 + t]] = static_cast<int32_t>(t);
    }
  }
}

// First tile-class trade of every tile (tile i = weight offsets [i C, (i+1) C)),
// plus the end sentinel; one thread per tile-class trade.
__global__ void k_tile_first(const int64_t* __restrict__ tile_off, const int64_t* __restrict__ counts,
                             int32_t* __restrict__ tile_first) {
  const int64_t ntr = counts[0], total_w = counts[3];
  const int64_t ntiles = (total_w + kTileCap - 1) / kTileCap;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < ntr; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t cur = tile_off[k] / kTileCap;
    const int64_t prev = k ? tile_off[k - 1] / kTileCap : -1;
    for (int64_t i = prev + 1; i <= cur; ++i) tile_first[i] = static_cast<int32_t>(k);
    if (k == ntr - 1)
      for (int64_t i = cur + 1; i <= ntiles; ++i) tile_first[i] = static_cast<int32_t>(ntr);
  }
}

// ---------------------------------------------------------------- tile path

// Shared memory of the tile kernels is budgeted so that four 256-thread CTAs
// fit on an SM (228 KB, 1 KB reserved per CTA): the threshold kernel's
// TileShared + TileA must stay below 56 KB.
struct TileShared {              // per-trade data of the current tile
  int64_t b0[kTileTrades];
  int32_t t[kTileTrades];
  int32_t acnt[kTileTrades];    // |A_{u-v}| (phase A)
  int32_t flags[kTileTrades];   // bit0 deferred, bit1 has a dependent later trade
  int16_t du[kTileTrades], dv[kTileTrades], lofs[kTileTrades];
  int64_t first, base;
  int32_t ntr, nslots;
};

// Per-entry arrays of a tile (phase-specific layouts provide them).
struct TileEntries {
  int32_t* y;
  uint16_t* owner;
  KeyCtx* kc;        // per trade, filled only when non-null
};

__device__ __forceinline__ int tile_owner(const TileShared& sh, int e) {
  int lo = 0, hi = sh.ntr;   // last local trade with lofs <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sh.lofs[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// Set up tile `tile`: its trades and entries (y) in shared memory.  Returns
// false when the tile is empty.
__device__ bool tile_setup(const StepCtx& c, TileShared& sh, const TileEntries& te, const int32_t* list,
                           const int64_t* tile_off, const int32_t* tile_first, int64_t ntrades, int64_t total_w,
                           int64_t tile) {
  if (threadIdx.x == 0) {
    const int64_t a = tile_first[tile];
    const int64_t b = tile_first[tile + 1];
    sh.first = a;
    sh.ntr = static_cast<int32_t>(b - a);
    sh.base = a < ntrades ? tile_off[a] : 0;
    sh.nslots = static_cast<int32_t>((b < ntrades ? tile_off[b] : total_w) - sh.base);
  }
  __syncthreads();
  if (sh.ntr == 0) return false;
  for (int j = threadIdx.x; j < sh.ntr; j += blockDim.x) {
    const int64_t k = sh.first + j;
    const int32_t t = list[k];
    const TradeRows tr = trade_rows(c, t);
    sh.t[j] = t;
    if (te.kc) te.kc[j] = key_ctx(c, t);
    sh.b0[j] = tr.b0;
    sh.du[j] = static_cast<int16_t>(tr.du);
    sh.dv[j] = static_cast<int16_t>(tr.dv);
    sh.lofs[j] = static_cast<int16_t>(tile_off[k] - sh.base);
    sh.acnt[j] = 0;
    sh.flags[j] = 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < sh.nslots; e += blockDim.x) {
    const int k = tile_owner(sh, e);
    const int i = e - sh.lofs[k];
    if (i < sh.du[k] + sh.dv[k]) {
      te.owner[e] = static_cast<uint16_t>(k);
      if (te.y) te.y[e] = __ldcg(c.col + sh.b0[k] + i);
    } else {
      te.owner[e] = kNoOwner;
    }
  }
  __syncthreads();
  return true;
}

// Phase A for a tile of small trades, one thread per entry.  The 2x2 block
// matrices come from a hash keyed by (local trade, far trade), the
// |A_{u-v}|-th smallest key of every trade from a radix select with 4-bit
// digits that all trades of the tile run together.
struct TileA {
  KeyCtx kc[kTileTrades];                 // key parameters of each trade's graph
  uint64_t key[kTileSlots];               // full own key
  unsigned long long hash[kTileHash];     // (key+1) << 16 | flags
  union {
    uint32_t hist[kTileTrades * 8];       // 16 bins per trade, two 16-bit counters per word
    uint64_t thr_tb[kTileTrades];         // after the selection: threshold tie-break
  };
  uint64_t prefix[kTileTrades];           // radix-select prefix, then the threshold key
  int32_t y[kTileSlots];
  uint16_t owner[kTileSlots];
  uint8_t meta[kTileSlots];
  uint8_t far[kTileSlots];
  int16_t kk[kTileTrades];                // rank still sought (1-based; |D| <= 128)
  int8_t shift[kTileTrades];
};

static_assert(sizeof(TileShared) + sizeof(TileA) + 1024 <= 233472 / 4, "tile threshold kernel: 4 CTAs per SM");

__device__ __forceinline__ uint64_t tile_hkey(int k, int64_t s) {
  return ((static_cast<uint64_t>(k) << 31) | static_cast<uint64_t>(s)) + 1;
}
__device__ __forceinline__ uint32_t tile_hslot(uint64_t hk) {
  const uint32_t x = static_cast<uint32_t>(hk) * 0x9E3779B1u ^ static_cast<uint32_t>(hk >> 32) * 0x85EBCA6Bu;
  return x >> (32 - kTileHashLg);
}
__device__ void tile_hinsert(unsigned long long* h, uint64_t hk, uint32_t bit) {
  uint32_t s = tile_hslot(hk);
  const unsigned long long want = static_cast<unsigned long long>(hk) << 16;
  for (;;) {
    unsigned long long cur = h[s];
    if (cur == 0ull) {
      const unsigned long long prev = atomicCAS(&h[s], 0ull, want | bit);
      if (prev == 0ull) return;
      cur = prev;
    }
    if ((cur >> 16) == hk) {
      atomicOr(reinterpret_cast<unsigned int*>(&h[s]), bit);
      return;
    }
    s = (s + 1) & (kTileHash - 1);
  }
}
__device__ __forceinline__ int tile_hfind(const unsigned long long* h, uint64_t hk) {
  uint32_t s = tile_hslot(hk);
  for (;;) {
    const unsigned long long cur = h[s];
    if (cur == 0ull) return -1;
    if ((cur >> 16) == hk) return static_cast<int>(s);
    s = (s + 1) & (kTileHash - 1);
  }
}

// Tile order: round robin over the CTAs (`blocked` = 0), or each CTA a run of
// consecutive tiles (`blocked` = 1).  A trade defers when a trade it depends
// on has not published yet: in one large graph those are spread over all
// earlier indices, and round robin finishes them first; in a batch of small
// graphs they sit in the tiles just before, which a CTA running consecutive
// tiles has already done.
__global__ void __launch_bounds__(kTileThreads) k_phase_a_tile(StepCtx c, const int32_t* __restrict__ list,
                                                               const int64_t* __restrict__ tile_off,
                                                               const int32_t* __restrict__ tile_first,
                                                               const int64_t* __restrict__ counts, int blocked) {
  __shared__ TileShared sh;
  extern __shared__ __align__(16) char dsm[];
  TileA& ta = *reinterpret_cast<TileA*>(dsm);
  const int64_t ntrades = counts[0], total_w = counts[3];
  const int64_t ntiles = (total_w + kTileCap - 1) / kTileCap;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;   // tiles per CTA when blocked
  for (int64_t i = 0;; ++i) {
    if (blocked && i >= per) break;
    const int64_t tile = blocked ? blockIdx.x * per + i : blockIdx.x + i * gridDim.x;
    if (tile >= ntiles) break;
    for (int i = threadIdx.x; i < kTileHash; i += blockDim.x) ta.hash[i] = 0ull;
    if (!tile_setup(c, sh, TileEntries{ta.y, ta.owner, ta.kc}, list, tile_off, tile_first, ntrades, total_w,
                    tile))
      continue;
    const int E = sh.nslots;
    // entries into the hash: presence bit (row, column) per (trade, far trade)
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int k = ta.owner[e];
      if (k == kNoOwner) continue;
      const int32_t yy = ta.y[e];
      const int64_t s = yy >> 1;
      if (s == sh.t[k]) continue;
      const int r = (e - sh.lofs[k]) >= sh.du[k];
      tile_hinsert(ta.hash, tile_hkey(k, s), 1u << (2 * r + (yy & 1)));
    }
    __syncthreads();
    // block analysis, dependencies, keys
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int k = ta.owner[e];
      if (k == kNoOwner) continue;
      const int64_t t = sh.t[k], t2 = 2 * t;
      const int r = (e - sh.lofs[k]) >= sh.du[k];
      const int32_t yy = ta.y[e];
      const int64_t s = yy >> 1;
      const bool single = (t2 + 1 >= c.n);
      ta.far[e] = 0;
      if (s == t) {
        ta.meta[e] = static_cast<uint8_t>(r | kUV);
        continue;
      }
      const int slot = tile_hfind(ta.hash, tile_hkey(k, s));
      const uint32_t bits = static_cast<uint32_t>(ta.hash[slot]) & 15u;
      const int u0 = bits & 1, u1 = (bits >> 1) & 1, v0 = (bits >> 2) & 1, v1 = (bits >> 3) & 1;
      const int cu = u0 + u1, cv = v0 + v1;
      uint8_t m = static_cast<uint8_t>(r | (u0 << 4) | (u1 << 5) | (v0 << 6) | (v1 << 7));
      const bool multi = (bits & (bits - 1u)) != 0;   // two or more block edges (rare)
      if (multi && !single && s > t && s < c.T && (u0 + v0 == 1 || u1 + v1 == 1)) atomicOr(&sh.flags[k], 2);
      int col_now = yy & 1;
      int other = 0;   // a single edge leaves the other row without this neighbour
      if (multi) other = r ? (col_now ? u1 : u0) : (col_now ? v1 : v0);
      if (multi && !single && s < t && (cu == 1 || cv == 1)) {
        if (ld_acquire(c.done + s) != c.stamp) {
          atomicOr(&sh.flags[k], 1);
          continue;
        }
        int m1[2][2] = {{0, 0}, {0, 0}};
        const int bb[2][2] = {{u0, u1}, {v0, v1}};
        const int cnt_row[2] = {cu, cv};
#pragma unroll
        for (int rho = 0; rho < 2; ++rho)
#pragma unroll
          for (int gam = 0; gam < 2; ++gam) {
            if (!bb[rho][gam]) continue;
            int g2 = gam;
            if (cnt_row[rho] == 1) {
              const uint32_t x = static_cast<uint32_t>(t2 + rho), y = static_cast<uint32_t>(2 * s + gam);
              g2 = far_keeps_low(c, ta.kc[k], s, min(x, y), max(x, y)) ? 0 : 1;
            }
            m1[rho][g2] = 1;
            if (rho == r && gam == (yy & 1)) col_now = g2;
          }
        other = m1[1 - r][col_now];
      }
      const uint32_t x = static_cast<uint32_t>(t2 + r), y = static_cast<uint32_t>(yy);
      const uint32_t lo = min(x, y), hi = max(x, y);
      const EdgeKeys ek = edge_keys(ta.kc[k], lo, hi);
      const bool lo_mine = (lo >> 1) == static_cast<uint32_t>(t);
      ta.key[e] = lo_mine ? ek.lo_side : ek.hi_side;
      ta.far[e] = static_cast<uint8_t>((lo_mine ? ek.hi_side : ek.lo_side) >> 58);
      if (!other && !single) {
        m |= kInD;
        if (r == 0) atomicAdd(&sh.acnt[k], 1);
      }
      ta.meta[e] = m;
    }
    __syncthreads();
    // deferred trades leave; the others start selecting their a-th smallest key
    for (int k = threadIdx.x; k < sh.ntr; k += blockDim.x) {
      const int32_t t = sh.t[k];
      if (sh.flags[k] & 1) {
        c.done[t] = kDeferred;
        atomicAdd(c.def_count, 1ull);
      }
      const bool skip = (sh.flags[k] & 1) || sh.acnt[k] == 0 || 2 * int64_t(t) + 1 >= c.n;
      ta.kk[k] = static_cast<int16_t>(skip ? 0 : sh.acnt[k]);
      ta.shift[k] = skip ? -1 : 60;
      ta.prefix[k] = 0;
    }
    __syncthreads();
    for (int round = 0; round < 16; ++round) {
      for (int i = threadIdx.x; i < kTileTrades * 8; i += blockDim.x) ta.hist[i] = 0;
      __syncthreads();
      for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int k = ta.owner[e];
        if (k == kNoOwner || !(ta.meta[e] & kInD)) continue;
        const int sft = ta.shift[k];
        if (sft < 0) continue;
        const uint64_t key = ta.key[e];
        if (sft < 60 && (key >> (sft + 4)) != (ta.prefix[k] >> (sft + 4))) continue;
        const uint32_t d = static_cast<uint32_t>(key >> sft) & 15u;
        atomicAdd(&ta.hist[k * 8 + (d >> 1)], (d & 1) ? 0x10000u : 1u);
      }
      __syncthreads();
      bool more = false;
      for (int k = threadIdx.x; k < sh.ntr; k += blockDim.x) {
        const int sft = ta.shift[k];
        if (sft < 0) continue;
        int below = 0;
        const int kk = ta.kk[k];
        for (int b = 0; b < 16; ++b) {
          const uint32_t w = ta.hist[k * 8 + (b >> 1)];
          const int cb = static_cast<int>((b & 1) ? (w >> 16) : (w & 0xffffu));
          if (below < kk && kk <= below + cb) {
            ta.kk[k] = static_cast<int16_t>(kk - below);
            ta.prefix[k] |= static_cast<uint64_t>(b) << sft;
            if (cb == 1 || sft == 0) {
              ta.shift[k] = static_cast<int8_t>(-2 - sft);   // resolved; -2 - shift keeps the last shift
            } else {
              ta.shift[k] = static_cast<int8_t>(sft - 4);
              more = true;
            }
            break;
          }
          below += cb;
        }
      }
      if (!__syncthreads_or(more)) break;   // every thread takes the same exit
    }
    for (int k = threadIdx.x; k < kTileTrades; k += blockDim.x) ta.thr_tb[k] = 0;   // histogram no longer needed
    __syncthreads();
    // the threshold element of each trade: the one matching its prefix (ties on
    // all 64 bits, which need the (lo, hi) order, are ranked explicitly)
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int k = ta.owner[e];
      if (k == kNoOwner || !(ta.meta[e] & kInD)) continue;
      const int code = ta.shift[k];
      if (code > -2) continue;
      const int sft = -2 - code;
      const uint64_t key = ta.key[e];
      if ((key >> sft) != (ta.prefix[k] >> sft)) continue;
      const int64_t t2 = 2 * static_cast<int64_t>(sh.t[k]);
      const uint8_t m = ta.meta[e];
      const uint64_t tb = tie_break(lo_of(t2, m, ta.y[e]), hi_of(t2, m, ta.y[e]));
      if (sft > 0) {
        ta.prefix[k] = key;
        ta.thr_tb[k] = tb;
      } else {   // every candidate has this exact key
        const int lo0 = sh.lofs[k], L = sh.du[k] + sh.dv[k];
        int r = 0;
        for (int j = lo0; j < lo0 + L; ++j) {
          if (j == e || !(ta.meta[j] & kInD) || ta.key[j] != key) continue;
          r += tie_break(lo_of(t2, ta.meta[j], ta.y[j]), hi_of(t2, ta.meta[j], ta.y[j])) < tb;
        }
        if (r == ta.kk[k] - 1) ta.thr_tb[k] = tb;
      }
    }
    __syncthreads();
    // own decisions; flips go into the hash for the far-side test
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int k = ta.owner[e];
      if (k == kNoOwner || (sh.flags[k] & 1)) continue;
      const uint8_t m = ta.meta[e];
      if (!(m & kInD)) continue;
      const int64_t t2 = 2 * static_cast<int64_t>(sh.t[k]);
      const int r = m & kR;
      const bool has_thr = ta.shift[k] <= -2;
      const bool low = has_thr && at_or_below(ta.key[e], tie_break(lo_of(t2, m, ta.y[e]), hi_of(t2, m, ta.y[e])),
                                              ta.prefix[k], ta.thr_tb[k]);
      if ((low ? 0 : 1) != r) {
        ta.meta[e] = m | kFlip;
        const int32_t yy = ta.y[e];
        const int slot = tile_hfind(ta.hash, tile_hkey(k, yy >> 1));
        atomicOr(reinterpret_cast<unsigned int*>(&ta.hash[slot]), 16u << (2 * r + (yy & 1)));
      }
    }
    __syncthreads();
    // will the far trade consider this edge?  Write the stash byte.
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int k = ta.owner[e];
      if (k == kNoOwner || (sh.flags[k] & 1)) continue;
      const uint8_t m = ta.meta[e];
      const int f = (m & kFlip) ? 1 : 0;
      int in_far = 0;
      const int64_t t = sh.t[k];
      if (!(m & kUV)) {
        const int r = m & kR;
        const int32_t yy = ta.y[e];
        const int64_t s = yy >> 1;
        const int u0 = (m >> 4) & 1, u1 = (m >> 5) & 1, v0 = (m >> 6) & 1, v1 = (m >> 7) & 1;
        const int cr = r ? (v0 + v1) : (u0 + u1);
        if (2 * t + 1 >= c.n || s < t) {
          in_far = (cr == 1);
        } else if (s < c.T) {
          if (u0 + u1 + v0 + v1 == 1) {
            in_far = 1;
          } else {   // block after t's own decisions: presence bits 0..3, flips 4..7
            const uint32_t fl = static_cast<uint32_t>(ta.hash[tile_hfind(ta.hash, tile_hkey(k, s))]);
            const int myrow = r ^ f;
            int same = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (!((fl >> q) & 1)) continue;
              same += (((q >> 1) ^ ((fl >> (4 + q)) & 1)) == myrow);
            }
            in_far = (same == 1);
          }
        }
      }
      c.stash[sh.b0[k] + (e - sh.lofs[k])] =
          static_cast<uint8_t>(f | (in_far << 1) | (in_far ? (ta.far[e] << 2) : 0));
    }
    // publish every completed trade's threshold (fenced when a later trade waits on it)
    for (int k = threadIdx.x; k < sh.ntr; k += blockDim.x) {
      const int32_t t = sh.t[k];
      if ((sh.flags[k] & 1) || 2 * int64_t(t) + 1 >= c.n) continue;
      const bool has_thr = ta.shift[k] <= -2;
      const uint64_t tk = has_thr ? ta.prefix[k] : 0;
      c.thr_key[t] = tk;
      c.thr_tb[t] = has_thr ? ta.thr_tb[k] : 0;
      c.thr_top[t] = static_cast<uint8_t>(tk >> 58);
      if (sh.flags[k] & 2) {
        __threadfence();
        st_release(c.done + t, c.stamp);
      }
    }
    __syncthreads();
  }
}

// --------------------------------------------------------- flat rebuild
//
// Phase B over the whole position-space adjacency at once: a CTA takes a
// chunk of 2048 consecutive entries, each thread 8 consecutive entries.  Trade
// t owns entries [rp[2t], rp[2t+2]); the trades a chunk touches go to a
// shared table (start, u/v boundary, new row offsets), or are looked up in
// global memory when a chunk spans more trades than the table holds (only
// with many empty trades).  Entries of the same (trade, new side) in a warp
// claim their slots together with one global atomic on the trade's counter
// (rows are sets; a counter past the row's degree latches an error).

constexpr int kFlatThreads = 256;
constexpr int kFlatPer = 8;                              // consecutive entries per thread
constexpr int kFlatChunk = kFlatThreads * kFlatPer;      // entries per chunk
constexpr int kFlatTrades = 512;                         // trades in the shared table

struct FlatTrade {
  int64_t start, b1;    // first entry, first entry of v's row
  int64_t ou, ov;       // new row offsets of u and v
  int32_t du, dv;
};

__device__ __forceinline__ FlatTrade flat_trade(const StepCtx& c, int64_t t) {
  FlatTrade f;
  f.start = c.rp[2 * t];
  f.b1 = c.rp[2 * t + 1];
  const bool single = 2 * t + 1 >= c.n;
  const int64_t end = single ? f.b1 : c.rp[2 * t + 2];
  f.du = static_cast<int32_t>(f.b1 - f.start);
  f.dv = static_cast<int32_t>(end - f.b1);
  const int32_t pu = c.M[2 * t];
  f.ou = c.rp_next[pu];
  bool bad = c.rp_next[pu + 1] - f.ou != f.du;
  f.ov = 0;
  if (!single) {
    const int32_t pv = c.M[2 * t + 1];
    f.ov = c.rp_next[pv];
    bad |= c.rp_next[pv + 1] - f.ov != f.dv;
  }
  if (bad) latch(c.err, kErrRowLength);
  return f;
}

// Last trade in [lo, hi] whose first entry is <= e (global row offsets).
__device__ __forceinline__ int64_t flat_owner(const StepCtx& c, int64_t lo, int64_t hi, int64_t e) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (c.rp[2 * mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// What the rebuild needs of a far trade s, in one record: the new positions
// of its two nodes and the top 6 bits of its threshold key.  Up to 2^29
// positions it fits 8 bytes (29 + 29 + 6 bits), else 16.
constexpr int64_t kNarrowPackMax = int64_t(1) << 29;

struct FarTrade {
  int32_t x, y;    // new positions of nodes 2s and 2s+1
  uint32_t top;    // threshold prefix
};

template <bool kNarrow>
__global__ void k_far_pack(StepCtx c, int64_t ntasks, void* __restrict__ pack) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < ntasks; s += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t x = static_cast<uint32_t>(c.M[2 * s]);
    const uint32_t y = 2 * s + 1 < c.n ? static_cast<uint32_t>(c.M[2 * s + 1]) : 0u;
    const uint32_t top = c.thr_top[s];
    if constexpr (kNarrow) {
      static_cast<uint64_t*>(pack)[s] = uint64_t(x) | (uint64_t(y) << 29) | (uint64_t(top) << 58);
    } else {
      static_cast<int4*>(pack)[s] = make_int4(static_cast<int32_t>(x), static_cast<int32_t>(y),
                                              static_cast<int32_t>(top), 0);
    }
  }
}

template <bool kNarrow>
__device__ __forceinline__ FarTrade far_trade(const void* pack, int32_t s) {
  if constexpr (kNarrow) {
    const uint64_t v = __ldg(static_cast<const unsigned long long*>(pack) + s);
    return {static_cast<int32_t>(v & 0x1FFFFFFFu), static_cast<int32_t>((v >> 29) & 0x1FFFFFFFu),
            static_cast<uint32_t>(v >> 58)};
  } else {
    const int4 v = __ldg(static_cast<const int4*>(pack) + s);
    return {v.x, v.y, static_cast<uint32_t>(v.z)};
  }
}

// The first and last trade with entries in each chunk (one thread per trade:
// every chunk boundary lies in exactly one non-empty trade).
__global__ void k_flat_ranges(StepCtx c, int64_t nnz, int64_t ntasks, int32_t* __restrict__ cf,
                              int32_t* __restrict__ cl) {
  const int64_t nchunks = (nnz + kFlatChunk - 1) / kFlatChunk;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < ntasks; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = c.rp[2 * t];
    const int64_t e = 2 * t + 1 >= c.n ? c.rp[2 * t + 1] : c.rp[2 * t + 2];
    if (e <= b) continue;
    // chunks whose first entry lies in [b, e)
    for (int64_t ch = (b + kFlatChunk - 1) / kFlatChunk; ch < nchunks && ch * kFlatChunk < e; ++ch)
      cf[ch] = static_cast<int32_t>(t);
    // chunks whose last entry lies in [b, e)
    for (int64_t ch = b / kFlatChunk; ch < nchunks; ++ch) {
      const int64_t last = ((ch + 1) * kFlatChunk < nnz ? (ch + 1) * kFlatChunk : nnz) - 1;
      if (last >= e) break;
      if (last >= b) cl[ch] = static_cast<int32_t>(t);
    }
  }
}

template <bool kNarrow>
__global__ void __launch_bounds__(kFlatThreads) k_phase_b_flat(StepCtx c, int64_t nnz, int64_t ntasks,
                                                               int32_t* __restrict__ slots,
                                                               const int32_t* __restrict__ cf,
                                                               const int32_t* __restrict__ cl,
                                                               const void* __restrict__ pack) {
  __shared__ FlatTrade tab[kFlatTrades];
  __shared__ int32_t cnt[2 * kFlatTrades];     // entries of this chunk per (local trade, new side)
  __shared__ int32_t gbase[2 * kFlatTrades];   // their first slot in the new row
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t nchunks = (nnz + kFlatChunk - 1) / kFlatChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t e0 = ch * kFlatChunk;
    const int64_t e1 = e0 + kFlatChunk < nnz ? e0 + kFlatChunk : nnz;
    const int64_t tf = cf[ch], tl = cl[ch];
    const int ntr = static_cast<int>(tl - tf + 1 < kFlatTrades + 1 ? tl - tf + 1 : kFlatTrades + 1);
    const bool in_table = ntr <= kFlatTrades;
    if (in_table) {
      for (int q = threadIdx.x; q < ntr; q += blockDim.x) tab[q] = flat_trade(c, tf + q);
      for (int q = threadIdx.x; q < 2 * ntr; q += blockDim.x) cnt[q] = 0;
    }
    __syncthreads();
    const int64_t base = e0 + static_cast<int64_t>(threadIdx.x) * kFlatPer;
    // owner of this thread's first entry, then walk forward
    int64_t q = 0;
    if (base < e1) {
      if (in_table) {
        int lo = 0, hi = ntr - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tab[mid].start <= base) lo = mid; else hi = mid - 1;
        }
        q = lo;
      } else {
        q = flat_owner(c, tf, tl, base) - tf;
      }
    }
    FlatTrade ft = in_table ? tab[q] : flat_trade(c, tf + q);
    int64_t next_start = (tf + q + 1 <= tl) ? (in_table ? tab[q + 1].start : c.rp[2 * (tf + q + 1)]) : INT64_MAX;
    // the thread's 8 entries and stash bytes (32 B and 8 B, aligned: chunks
    // start at multiples of 2048 entries); a partial run at the end loads singly
    int32_t yv[kFlatPer];
    uint8_t sv[kFlatPer];
    if (base + kFlatPer <= e1) {
      const int4 a0 = __ldcs(reinterpret_cast<const int4*>(c.col + base));
      const int4 a1 = __ldcs(reinterpret_cast<const int4*>(c.col + base) + 1);
      yv[0] = a0.x; yv[1] = a0.y; yv[2] = a0.z; yv[3] = a0.w;
      yv[4] = a1.x; yv[5] = a1.y; yv[6] = a1.z; yv[7] = a1.w;
      const uint2 b = __ldcs(reinterpret_cast<const uint2*>(c.stash + base));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sv[j] = static_cast<uint8_t>(b.x >> (8 * j));
        sv[4 + j] = static_cast<uint8_t>(b.y >> (8 * j));
      }
    } else {
#pragma unroll
      for (int j = 0; j < kFlatPer; ++j) {
        yv[j] = base + j < e1 ? c.col[base + j] : 0;
        sv[j] = base + j < e1 ? c.stash[base + j] : 0;
      }
    }
    int32_t outv[kFlatPer], keyv[kFlatPer], posv[kFlatPer];
#pragma unroll
    for (int j = 0; j < kFlatPer; ++j) {
      const int64_t e = base + j;
      const bool valid = e < e1;
      if (valid) {
        while (e >= next_start) {   // next non-empty trade (empty trades share its start)
          ++q;
          ft = in_table ? tab[q] : flat_trade(c, tf + q);
          next_start = (tf + q + 1 <= tl) ? (in_table ? tab[q + 1].start : c.rp[2 * (tf + q + 1)]) : INT64_MAX;
        }
      }
      int key = -1;
      int32_t out = 0;
      if (valid) {
        const int64_t t = tf + q;
        const int r = e >= ft.b1;
        const int32_t yy = yv[j];
        const uint8_t st = sv[j];
        const int r2 = r ^ (st & 1);
        const int32_t s = yy >> 1;
        const FarTrade fs = far_trade<kNarrow>(pack, s);   // one gather: new positions, threshold prefix
        int hi_node = yy & 1;
        if (st & 2) {
          const uint32_t fp = st >> 2, tt = fs.top;
          bool low;
          if (fp != tt) {
            low = fp < tt;
          } else {
            const uint32_t x = static_cast<uint32_t>(2 * t + r), y = static_cast<uint32_t>(yy);
            low = far_keeps_low(c, key_ctx(c, t), s, min(x, y), max(x, y));   // prefix tie: 1 in 64
          }
          hi_node = low ? 0 : 1;
        }
        out = hi_node ? fs.y : fs.x;
        key = static_cast<int>(2 * q + r2);
      }
      // the entries of one (trade, side) in the warp take consecutive slots
      const unsigned grp = __match_any_sync(kFull, key);
      const int leader = __ffs(grp) - 1;
      int slot0 = 0;
      if (lane == leader && key >= 0)
        slot0 = in_table ? atomicAdd(&cnt[key], __popc(grp))
                         : atomicAdd(&slots[2 * (tf + q) + (key & 1)], __popc(grp));
      slot0 = __shfl_sync(kFull, slot0, leader);
      outv[j] = out;
      keyv[j] = key;
      posv[j] = slot0 + __popc(grp & below);
      if (!in_table && key >= 0) {   // global slot already final
        const int p = posv[j];
        const int r2 = key & 1;
        if (p < (r2 ? ft.dv : ft.du)) c.col_next[(r2 ? ft.ov : ft.ou) + p] = out;
        else latch(c.err, kErrRowSide);
      }
    }
    if (in_table) {
      // one global reservation per (trade, side) of the chunk, then the writes
      __syncthreads();
      for (int k = threadIdx.x; k < 2 * ntr; k += blockDim.x)
        if (cnt[k]) gbase[k] = atomicAdd(&slots[2 * (tf + (k >> 1)) + (k & 1)], cnt[k]);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kFlatPer; ++j) {
        const int key = keyv[j];
        if (key < 0) continue;
        const FlatTrade& f = tab[key >> 1];
        const int r2 = key & 1;
        const int p = gbase[key] + posv[j];
        if (p < (r2 ? f.dv : f.du)) c.col_next[(r2 ? f.ov : f.ou) + p] = outv[j];
        else latch(c.err, kErrRowSide);
      }
    }
    __syncthreads();   // the table is reloaded for the next chunk
  }
}

// ---------------------------------------------------------------- team paths

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) k_phase_a_block(StepCtx c, const int32_t* __restrict__ list,
                                                      const int64_t* __restrict__ count, int smem_max, char* gws,
                                                      size_t slice, int stage_cap) {
  // dynamic shared memory: the workspace, then the staging buffer of a
  // trade's entries (stage_cap + 8 int32, 16-byte aligned)
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ SelOut sel;
  __shared__ uint64_t mbar;
  BlockTeam<NT> tm(red);
  const int64_t len = *count;
  int32_t* stage = reinterpret_cast<int32_t*>(sbuf + ((ws_a_bytes(smem_max) + 127) & ~size_t(127)));
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  // member 0 reads the next trade's row range at the start of each trade; the
  // copy goes out once the current trade has read its staged entries
  auto range_of = [&](int64_t q, int64_t* b0, int* L) {
    const int64_t t = list[q];
    const TradeRows tr = trade_rows(c, t);
    *b0 = tr.b0;
    *L = tr.du + tr.dv;
  };
  int64_t nb0 = 0;
  int nL = 0;
  // a trade is staged when it has entries and fits the buffer (every thread
  // applies the same test to the same trade)
  auto staged = [&](int L) { return L > 0 && L <= stage_cap; };
  if (threadIdx.x == 0 && blockIdx.x < len) {
    range_of(blockIdx.x, &nb0, &nL);
    if (staged(nL)) stage_issue(c.col, nb0, nL, stage, &mbar);
  }
  bool failed = false;
  for (int64_t q = blockIdx.x; q < len; q += gridDim.x) {
    const int64_t t = list[q];
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    char* base = sbuf;
    if (L > smem_max) {
      base = gws + slice * blockIdx.x;
      if (threadIdx.x == 0) atomicAdd(c.gws_count, 1ull);
    }
    StageNext sn{false, 0, 0, stage, &mbar};
    if (threadIdx.x == 0 && q + gridDim.x < len) {
      range_of(q + gridDim.x, &nb0, &nL);
      sn.issue = staged(nL);
      sn.b0 = nb0;
      sn.L = nL;
    }
    const int32_t* ys = nullptr;
    if (staged(L)) {   // this trade's entries were staged by the previous one (or the prologue)
      const bool late = !mbar_wait(&mbar, parity);
      parity ^= 1;
      if (__syncthreads_or(late)) {
        failed = true;
        break;
      }
      ys = stage + stage_off(tr.b0);
    }
    phase_a(tm, c, t, carve_a(base, L), &sel, ys, sn);
  }
  if (failed) {   // a copy did not complete in time: report, let it land, leave
    if (threadIdx.x == 0) latch(c.err, kErrStage);
    mbar_wait(&mbar, parity ^ 1);
  }
}

// The trades the first pass deferred, in index order.  CTAs claim chunks of
// trade indices in increasing order and run the deferred trades of a chunk one
// after another; a trade waits for an unpublished dependency instead of
// deferring.  A dependency s < t is either complete (first pass) or deferred
// too, and then it sits in an earlier chunk or earlier in the same chunk:
// claimed before t by a CTA that is already running.  By induction on the
// index, the smallest unfinished claimed trade waits for nothing, so every
// wait ends whatever the residency of the grid.
template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) k_phase_a_inorder(StepCtx c, int64_t ntasks, int64_t chunk,
                                                        unsigned long long* claim, int smem_max, char* gws,
                                                        size_t slice) {
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ SelOut sel;
  __shared__ int64_t first;
  __shared__ int32_t found[NT];
  __shared__ int nfound;
  BlockTeam<NT> tm(red);
  for (;;) {
    if (threadIdx.x == 0) first = static_cast<int64_t>(atomicAdd(claim, 1ull)) * chunk;
    __syncthreads();
    const int64_t lo = first;
    if (lo >= ntasks) return;
    const int64_t hi = lo + chunk < ntasks ? lo + chunk : ntasks;
    for (int64_t base = lo; base < hi; base += NT) {
      // the deferred trades of this slice of the chunk, in index order
      const int64_t t0 = base + threadIdx.x;
      const int mine = (t0 < hi && __ldcg(c.done + t0) == kDeferred) ? 1 : 0;
      const int before = static_cast<int>(tm.exscan(mine));
      if (mine) found[before] = static_cast<int32_t>(t0);
      if (threadIdx.x == NT - 1) nfound = before + mine;
      __syncthreads();
      const int nf = nfound;
      for (int q = 0; q < nf; ++q) {
        const int64_t t = found[q];
        const TradeRows tr = trade_rows(c, t);
        const int L = tr.du + tr.dv;
        char* wsb = sbuf;
        if (L > smem_max) {
          wsb = gws + slice * blockIdx.x;
          if (threadIdx.x == 0) atomicAdd(c.gws_count, 1ull);
        }
        phase_a(tm, c, t, carve_a(wsb, L), &sel);
      }
      __syncthreads();
    }
  }
}

// End of a super step: every graph's step counter moves on.
__global__ void k_seg_advance(Seg* segs, int nseg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += gridDim.x * blockDim.x) segs[i].g += 1;
}

int finish_step(Graph* h) {
  k_seg_advance<<<(h->nseg + 255) / 256, 256, 0, h->stream>>>(h->segs, h->nseg);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  h->cur = 1 - h->cur;
  h->g += 1;
  return CB_OK;
}

}  // namespace

int init_trade_kernels(Graph* h) {
  // the largest dynamic shared memory any handle may ask of each kernel
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kMedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(block_smem_bytes(kBlockMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(block_smem_bytes(kSmemMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_inorder<kMedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(ws_a_bytes(kBlockMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_inorder<kBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(ws_a_bytes(kSmemMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sizeof(TileA))));
  // shared memory, not L1, limits how many CTAs of these kernels an SM holds
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_tile, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kMedThreads>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  return CB_OK;
}

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
  c.stamp = 1;   // done flags are cleared at the start of every step
  c.segs = h->segs;
  c.seg_of = h->seg_of;
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
  // counters: [0..2] class list lengths, [3] tile weight total, [4..5] deferred
  // lists, [8..] pass input counts, [kCounters-1] global-workspace trades
  int64_t* cnt = h->counters;
  unsigned long long* ucnt = reinterpret_cast<unsigned long long*>(cnt);
  c.gws_count = ucnt + kCounters - 1;
  CB_CUDA(h, cudaMemsetAsync(cnt, 0, kCounters * sizeof(int64_t), s));
  const int64_t ntasks = h->ntasks;
  if (ntasks == 0) return finish_step(h);
  CB_CUDA(h, cudaMemsetAsync(h->done, 0, sizeof(uint32_t) * ntasks, s));
  const int tile_max = std::min(h->tile_max, kTileMaxCap);
  const int block_max = std::max(h->block_max, tile_max);
  auto grid_n = [&](int64_t work) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, h->num_sms * 8)));
  };
  {  // classes in index order (stable compaction) and tile offsets
    k_class_flags<<<grid_n(ntasks), 256, 0, s>>>(c, ntasks, tile_max, block_max, h->cls_flag);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    const int64_t n1 = ntasks + 1;
    for (int q = 0; q < 4; ++q)
      CB_CUDA(h, exclusive_scan_i32(h->cls_flag + q * ntasks, h->cls_scan + q * n1, ntasks, h->scan_ws, s,
                                    &h->launches));
    k_class_scatter<<<grid_n(ntasks), 256, 0, s>>>(ntasks, h->cls_flag, h->cls_scan, h->list[0], h->list[1],
                                                    h->list[2], h->tile_off);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    for (int q = 0; q < 4; ++q)
      CB_CUDA(h, cudaMemcpyAsync(cnt + q, h->cls_scan + q * n1 + ntasks, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_tile_first<<<grid_n(ntasks), 256, 0, s>>>(h->tile_off, cnt, h->tile_first);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  }
  const size_t med_smem = ws_a_bytes(std::max(block_max, 1));      // in-order pass (no staging)
  const size_t big_smem = ws_a_bytes(std::max(h->smem_max, 1));
  const size_t med_smem_st = block_smem_bytes(std::max(block_max, 1));   // threshold kernels with staging
  const size_t big_smem_st = block_smem_bytes(std::max(h->smem_max, 1));
  const unsigned tgrid = static_cast<unsigned>(h->num_sms * 8);
  const unsigned mgrid = static_cast<unsigned>(h->num_sms * 4);
  const unsigned bgrid = static_cast<unsigned>(std::max(1, std::min(h->num_sms, h->ws_ctas)));
  char* gws = static_cast<char*>(h->ws_global);
  // phase A, first pass: every class; a trade whose dependency has not
  // published yet is marked deferred.  Counters: [4] deferred trades, [5]
  // chunks claimed by the in-order pass.
  c.wait = 0;
  c.def_count = ucnt + 4;
  if (h->tile_paths & 1) {
    k_phase_a_tile<<<tgrid, kTileThreads, sizeof(TileA), s>>>(c, h->list[0], h->tile_off, h->tile_first, cnt,
                                                              h->nseg > 1 ? 1 : 0);
  } else {
    k_phase_a_block<kMedThreads><<<mgrid, kMedThreads, med_smem_st, s>>>(c, h->list[0], cnt + 0, block_max, gws,
                                                                        h->ws_slice, block_max);
  }
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_a_block<kMedThreads><<<mgrid, kMedThreads, med_smem_st, s>>>(c, h->list[1], cnt + 1, block_max, gws,
                                                                      h->ws_slice, block_max);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  k_phase_a_block<kBigThreads><<<bgrid, kBigThreads, big_smem_st, s>>>(c, h->list[2], cnt + 2, h->smem_max, gws,
                                                                      h->ws_slice, h->smem_max);
  CB_CUDA(h, cudaGetLastError());
  ++h->launches;
  // second pass: the deferred trades in index order, waiting on dependencies.
  // 1024-thread CTAs keep large trades in shared memory; 256-thread CTAs (four
  // per SM) run many small deferred trades at once, large ones from a global
  // slice.
  c.wait = 1;
  if (h->inorder_threads == kBigThreads) {
    const int64_t chunk = std::max<int64_t>(1024, (ntasks + int64_t(bgrid) * 8 - 1) / (int64_t(bgrid) * 8));
    k_phase_a_inorder<kBigThreads><<<bgrid, kBigThreads, big_smem, s>>>(c, ntasks, chunk, ucnt + 5, h->smem_max, gws,
                                                                       h->ws_slice);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  } else {
    const unsigned igrid = static_cast<unsigned>(gws ? std::min(h->num_sms * 4, h->ws_ctas) : h->num_sms * 4);
    const int64_t chunk = std::max<int64_t>(512, (ntasks + int64_t(igrid) * 4 - 1) / (int64_t(igrid) * 4));
    k_phase_a_inorder<kMedThreads><<<igrid, kMedThreads, med_smem, s>>>(c, ntasks, chunk, ucnt + 5, block_max, gws,
                                                                       h->ws_slice);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
  }
  if (h->timing) CB_CUDA(h, cudaEventRecord(h->ev[2], s));
  // phase B: one flat pass over every entry; per-trade slot counters start at zero
  {
    int32_t* slots = h->cls_flag;   // 2 x ntasks, free after the classification
    int32_t* cf = h->cls_flag + 2 * ntasks;   // chunk ranges (the scratch holds 2 x (nnz / 2048 + 1) more)
    const int64_t nchunks = (h->nnz + kFlatChunk - 1) / kFlatChunk;
    int32_t* cl = cf + nchunks;
    CB_CUDA(h, cudaMemsetAsync(slots, 0, sizeof(int32_t) * 2 * ntasks, s));
    if (nchunks > 0) {
      k_flat_ranges<<<grid_n(ntasks), 256, 0, s>>>(c, h->nnz, ntasks, cf, cl);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
      const bool narrow = h->n <= kNarrowPackMax && !h->wide_pack;
      if (narrow) k_far_pack<true><<<grid_n(ntasks), 256, 0, s>>>(c, ntasks, h->far_pack);
      else k_far_pack<false><<<grid_n(ntasks), 256, 0, s>>>(c, ntasks, h->far_pack);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
      const unsigned fgrid = static_cast<unsigned>(std::min<int64_t>(nchunks, int64_t(h->num_sms) * 8));
      if (narrow) k_phase_b_flat<true><<<fgrid, kFlatThreads, 0, s>>>(c, h->nnz, ntasks, slots, cf, cl, h->far_pack);
      else k_phase_b_flat<false><<<fgrid, kFlatThreads, 0, s>>>(c, h->nnz, ntasks, slots, cf, cl, h->far_pack);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
    }
  }
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
  return finish_step(h);
}

}  // namespace cb
