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
//  A. Threshold and placement.  Every trade finds
//     D = (A_u u A_v) \ (A_u n A_v) \ {u, v} (Def. "Simple Undirected Trade"),
//     keys its elements and publishes the threshold (key, lo, hi) of its
//     |A_{u-v}|-th smallest element: u keeps exactly the elements at or below
//     it (Fig. 2: u receives the first |A_{u-v}| elements of sigma(D)).  In
//     the same pass it places every entry in the row of its node after the
//     trade (step g+1 layout): the far end's step-g position as a placeholder,
//     and a 16-bit side word (bit 0 the own trade's flip, bits 1..11 the top
//     11 bits of the far trade's key for the edge, bit 12 set when the far
//     trade decides the edge).  The first pass runs every trade by size
//     class; a trade whose dependency has not published is deferred and
//     listed, retry passes run the lists, and one in-order pass completes
//     what is left, waiting (bounded) for its dependencies.
//  B. Rebuild (fix-up).  Every placeholder becomes the step-(g+1) position
//     of the far end: per far trade one packed record (the new positions of
//     its two nodes, the top 8 bits of its threshold), read in slices small
//     enough to stay in L2; the 8-bit prefix decides, then the 11-bit one,
//     and only on a tie there the full key.
//
// Phase A by trade size L = deg u + deg v (nine classes): lane teams of 8 or
// 16 threads (several trades per warp) and whole warps up to `tile_max`
// entries, teams of 64 to 1024 threads with the entries in registers up to
// min(4096, `smem_max`), and a 1024-thread CTA with the entries in shared
// memory (a global-memory slice above `smem_max`) for the largest.  The team
// and shared-memory kernels come in a version for handles of one graph,
// whose seed's Philox round keys are kernel parameters, and a general one.
#include <algorithm>
#include <type_traits>

#include "cb_internal.cuh"
#include "philox.cuh"
#include "team.cuh"

namespace cb {
namespace {

constexpr uint32_t kDeferred = 2;              // done[t]: deferred (a dependency had not published)
constexpr uint32_t kComplete = 3;              // done[t]: complete, no later trade waits for it

// meta bits per entry (phase A)
constexpr uint8_t kR = 1;       // entry sits in v's row
constexpr uint8_t kInD = 2;     // element of D_t
constexpr uint8_t kFlip = 4;    // trade t moves the edge to its other node
constexpr uint8_t kUV = 8;      // the edge {u_t, v_t}
// (kCol and kPend below: the neighbour's column, not hashed yet)

constexpr int kMedThreads = 256;
constexpr int kBigThreads = 1024;

struct StepCtx {
  int64_t n, T;
  uint32_t stamp;
  const Seg* segs;          // per graph: seed, step, first position
  const int32_t* seg_of;    // graph of each position (null: one graph)
  const int64_t* rp;
  const int32_t* col;
  uint16_t* fb;             // side word of every placed entry (step g+1 layout)
  int32_t* ph;              // placeholders of every entry in its new row (step g+1 layout)
  const int32_t* Minv;      // step-(g+1) position -> step-g position
  uint64_t* thr_key;
  uint64_t* thr_tb;
  uint8_t* thr_top;
  uint32_t* done;
  int32_t* err;
  const int32_t* M;
  const int64_t* rp_next;
  unsigned long long* def_count;   // trades this pass deferred
  int32_t* def_list;               // where they go (null: not listed): trades of at most kListSmall
  unsigned long long* def_small;   // entries from position 0 up, the others from def_cap - 1 down,
  unsigned long long* def_big;     // counted here
  int64_t def_cap;
  uint32_t wait;                   // 0: defer a trade whose dependency is unpublished; 1: wait for it
  unsigned long long* gws_count;
  int cand_max;                    // register paths: most candidates ranked directly (else more radix digits)
  uint64_t wait_ns;                // longest single wait on a dependency or a bulk copy
  int hold_publish;                // test hook: no trade publishes its done flag (waits run out)
  uint32_t ks[20];                 // one graph (seg_of null): the Philox round keys of its seed
};

struct SelOut {
  uint64_t key, tb;
  int32_t bin, below, cnt, pad;
};

// The trades of class k: (list, length).
struct ClassList {
  const int32_t* list;
  int64_t len;
};
__device__ __forceinline__ ClassList class_list(const int32_t* lists, const int64_t* ctr, int k) {
  return {lists + ctr[kCtrClsStart + k], ctr[kCtrClsLen + k]};
}

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
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// A trade whose dependency has not published: marked, counted, and listed
// for the next pass, small trades (L <= kListSmall, run on warps) apart from
// the others.
constexpr int kListSmall = 128;
__device__ __forceinline__ void defer_trade(const StepCtx& c, int64_t t, int L) {
  c.done[t] = kDeferred;
  atomicAdd(c.def_count, 1ull);
  if (!c.def_list) return;
  if (L <= kListSmall) {
    c.def_list[atomicAdd(c.def_small, 1ull)] = static_cast<int32_t>(t);
  } else {
    c.def_list[c.def_cap - 1 - static_cast<int64_t>(atomicAdd(c.def_big, 1ull))] = static_cast<int32_t>(t);
  }
}

// In-order passes: wait until trade s has published (true), at most wait_ns;
// a wait that runs out latches kErrResolve, and after any error every wait
// gives up at once (false).
__device__ __noinline__ bool wait_published(const uint32_t* done_s, int32_t* err, uint32_t stamp, uint64_t wait_ns) {
  const uint64_t t0 = globaltimer();
  while (ld_acquire(done_s) != stamp) {
    if (ld_volatile_i32(err) != 0) return false;
    if (globaltimer() - t0 > wait_ns) {
      latch(err, kErrResolve);
      return false;
    }
    __nanosleep(128);
  }
  return true;
}

// ------------------------------------------------- bulk copies (TMA engine)
//
// A trade's entries are staged into shared memory by one cp.async.bulk copy
// that completes on an mbarrier.  The copy moves whole 16-byte units, so it
// starts at the entry rounded down to a multiple of 4 and covers a multiple
// of 4 entries; the adjacency buffers carry 16 spare entries at their end, so
// the copy never leaves its allocation.


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
// sleep, at most wait_ns); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, uint64_t wait_ns) {
  if (mbar_test_wait(m, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    __nanosleep(64);
    if (mbar_test_wait(m, parity)) return true;
    if (globaltimer() - t0 > wait_ns) return false;
  }
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
// kOneSeed: a handle of one graph, whose seed's round keys are c.ks.
struct EdgeKeys {
  uint64_t lo_side, hi_side;
};
template <bool kOneSeed>
__device__ __forceinline__ EdgeKeys edge_keys(const StepCtx& c, const KeyCtx& kc, uint32_t lo, uint32_t hi) {
  Philox4 r;
  if constexpr (kOneSeed) {
    r = philox4x32_10_rk(lo - kc.off, hi - kc.off, kc.g, 1u, c.ks);
  } else {
    r = philox4x32_10(lo - kc.off, hi - kc.off, kc.g, 1u, kc.seed);
  }
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

// Slot of key (far trade + 1) starting the probe at p: the key's slot if an
// entry of the same far trade placed it, else the first empty slot, claimed
// with a compare-and-swap.  Used only for the few entries that lost the
// plain-store round of an insert.
__device__ __forceinline__ uint32_t h_claim(uint32_t* hk, uint32_t mask, uint32_t key, uint32_t p) {
  for (;;) {
    uint32_t cur = hk[p];
    if (cur == 0u) {
      cur = atomicCAS(&hk[p], 0u, key);
      if (cur == 0u) return p;
    }
    if (cur == key) return p;
    p = (p + 1u) & mask;
  }
}

// ---------------------------------------------------------- workspace

constexpr int kSelBits = 10;              // first radix digit: top 10 bits of the key
constexpr int kSelBins = 1 << kSelBits;

// meta bits per entry (team paths add the neighbour's column bit)
constexpr uint8_t kCol = 16;    // neighbour sits at the odd position 2s+1
constexpr uint8_t kPend = 32;   // not placed in the hash yet
// Bits of the far trade's key an entry's side word keeps (the rebuild decides
// with them unless they equal the far threshold's, 1 in 2^kFarBits).
constexpr int kFarBits = 11;
// Placeholder and side-word bits (see the rebuild's fix-up).
constexpr uint32_t kPhDone = 0x80000000u;   // placeholder resolved by an earlier pass (new position in bits 0..30)
constexpr uint32_t kFbInFar = 1u << 12;     // side word: the far trade decides the edge

constexpr int kCand = 32;       // candidates sharing the threshold's bin, ranked by full key

struct WsA {
  uint64_t* ck;               // kCand candidate keys
  uint64_t* ctb;              // their tie-breaks
  int32_t* cidx;              // their entry indices
  int32_t* ncand;
  int32_t* slot;              // hash slot of the entry's far trade (-1: the edge {u,v})
  uint16_t* top;              // top 16 bits of the own key
  uint8_t* meta;
  uint16_t* far;              // top kFarBits bits of the far trade's key
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
  return H * 4 + ((H + 15) & ~size_t(15)) + kSelBins * 4 + kCand * 20 + 16 + L16 * 4 + L16 * 2 + L16 + L16 * 2 + 64;
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
  w.far = reinterpret_cast<uint16_t*>(p);
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

template <class Team, bool kOneSeed = false>
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
  // entries into the hash: the far trade's slot (open addressing, far trade
  // + 1 as key: a plain store into an empty home slot, read back after a
  // barrier; an entry whose home slot another key won claims a further slot
  // with a compare-and-swap), then the presence bit (row, column) in the
  // slot's flags
  for (int i = tm.rank; i < L; i += Team::N) {
    const int r = i >= du;
    const int32_t yy = ystage ? ystage[i] : __ldcg(c.col + tr.b0 + i);
    const int64_t s = yy >> 1;
    uint8_t m = static_cast<uint8_t>(r | ((yy & 1) ? kCol : 0));
    if (s == t) {
      m |= kUV;
      w.slot[i] = -1;
    } else {
      m |= kPend;
      w.slot[i] = static_cast<int32_t>(hslot(static_cast<uint32_t>(s), w.lgH));
    }
    w.meta[i] = m;
  }
  {
    const uint32_t hmask = (1u << w.lgH) - 1u;
    for (int i = tm.rank; i < L; i += Team::N) {
      if (!(w.meta[i] & kPend)) continue;
      const int32_t yy = ystage ? ystage[i] : __ldcg(c.col + tr.b0 + i);
      const int sl = w.slot[i];
      if (w.hkey[sl] == 0u) w.hkey[sl] = (static_cast<uint32_t>(yy) >> 1) + 1u;
    }
    tm.sync();
    for (int i = tm.rank; i < L; i += Team::N) {
      const uint8_t m = w.meta[i];
      if (!(m & kPend)) continue;
      const int32_t yy = ystage ? ystage[i] : __ldcg(c.col + tr.b0 + i);
      const uint32_t sl = static_cast<uint32_t>(w.slot[i]);
      const uint32_t key = (static_cast<uint32_t>(yy) >> 1) + 1u;
      if (w.hkey[sl] != key)   // lost the slot to another key: claim one further on
        w.slot[i] = static_cast<int32_t>(h_claim(w.hkey, hmask, key, (sl + 1u) & hmask));
      w.meta[i] = m & ~kPend;
    }
    tm.sync();
    for (int i = tm.rank; i < L; i += Team::N) {
      const uint8_t m = w.meta[i];
      if (m & kUV) continue;
      flag_or(w.hflag, w.slot[i], 1u << (2 * (m & kR) + ((m & kCol) ? 1 : 0)));
    }
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
          // earlier, so the wait ends; the time limit turns a broken invariant
          // into an error, after which every other wait gives up at once
          const uint64_t t0 = globaltimer();
          while (ld_acquire(c.done + s) != c.stamp) {
            if (ld_volatile_i32(c.err) != 0) break;
            if (globaltimer() - t0 > c.wait_ns) {
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
    const EdgeKeys ek = edge_keys<kOneSeed>(c, kc, lo, hi);
    const bool lo_mine = (lo >> 1) == t32;
    const uint32_t top = static_cast<uint32_t>((lo_mine ? ek.lo_side : ek.hi_side) >> 48);
    w.top[i] = static_cast<uint16_t>(top);
    w.far[i] = static_cast<uint16_t>((lo_mine ? ek.hi_side : ek.lo_side) >> (64 - kFarBits));
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
    if (tm.rank == 0) defer_trade(c, t, L);
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
  // placement: each entry goes into the new row of its node after the trade
  // (u's or v's row of step g+1) at a slot given by a scan over the team
  int n0 = 0, n1 = 0;
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    const int side = (m & kR) ^ ((m & kFlip) ? 1 : 0);
    n0 += side == 0;
    n1 += side;
  }
  const int64_t pre = tm.exscan(static_cast<int64_t>(n0) | (static_cast<int64_t>(n1) << 32));
  int s0 = static_cast<int>(pre & 0xffffffff), s1 = static_cast<int>(pre >> 32);
  if (tm.rank == Team::N - 1 && (s0 + n0 != du || s1 + n1 != dv)) latch(c.err, kErrRowLength);
  const int64_t ou = c.rp_next[c.M[2 * t]];
  const int64_t ov = tr.single ? 0 : c.rp_next[c.M[2 * t + 1]];
  for (int i = tm.rank; i < L; i += Team::N) {
    const uint8_t m = w.meta[i];
    const int f = (m & kFlip) ? 1 : 0;
    int in_far = 0;
    if (!(m & kUV)) {   // will the far trade decide this edge?
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
    const int side = (m & kR) ^ f;
    const int k = side ? s1++ : s0++;
    if (k >= (side ? dv : du)) continue;   // counts checked above: never write outside the row
    const int64_t slot = (side ? ov : ou) + k;
    c.ph[slot] = entry_y(w, t2, i);
    c.fb[slot] = static_cast<uint16_t>(f | (in_far ? ((w.far[i] << 1) | kFbInFar) : 0u));
  }
  if (tm.rank == 0 && !tr.single) {
    c.thr_key[t] = tk;
    c.thr_tb[t] = tt;
    c.thr_top[t] = static_cast<uint8_t>(tk >> 56);
    if (publish_fence && !c.hold_publish) {
      __threadfence();
      st_release(c.done + t, c.stamp);
    } else if (!publish_fence) {
      c.done[t] = kComplete;   // a deferred trade done in a retry pass leaves the deferred list
    }
  }
  tm.sync();
}

// ------------------------------------------------ register-resident phase A
//
// The same decisions as phase_a for a trade whose L = deg u + deg v entries
// fit the team's registers (J entries per member, entry i held by member
// i mod N): each member keeps its entries' neighbour positions, key bits and
// flags in registers across the passes, so the only shared-memory traffic is
// the far-trade hash, one histogram and the few candidates of the threshold's
// bin.  Used by the first pass only: a trade whose dependency has not
// published yet is deferred to the in-order pass.

// per-entry meta word
constexpr uint32_t kMSlot = 0x3FFFu;        // hash slot of the far trade (tables of at most 2^14 slots)
constexpr uint32_t kMR = 1u << 14;          // entry sits in v's row
constexpr uint32_t kMCol = 1u << 15;        // neighbour at the odd position 2s+1
constexpr uint32_t kMUV = 1u << 16;         // the edge {u, v}
constexpr uint32_t kMInD = 1u << 17;        // element of D
constexpr uint32_t kMFlip = 1u << 18;       // the trade moves the edge to its other node
constexpr uint32_t kMValid = 1u << 19;      // an entry of the trade
constexpr uint32_t kMMulti = 1u << 20;      // block of two or more edges
constexpr int kMFarShift = 21;              // bits 21..31: top kFarBits bits of the far trade's key

__host__ __device__ constexpr int hash_lg_c(int L) {
  int lg = 1;
  while ((1 << lg) < 2 * L) ++lg;
  return lg;
}

// One team's workspace: a base address and a compile-time layout for trades
// of at most LMAX entries and 2^B histogram bins.
template <int LMAX, int B>
struct RegWs {
  static_assert(B >= 5, "tables are cleared in 16-byte stores");
  static constexpr int kLmax = LMAX;
  static constexpr int kH = 1 << hash_lg_c(2 * LMAX);   // at least 4 slots per entry
  static constexpr size_t kCk = 0;                              // candidate keys
  static constexpr size_t kCtb = kCk + kCand * 8;               // candidate tie-breaks
  static constexpr size_t kSel = kCtb + kCand * 8;              // selection results shared by the team
  static constexpr size_t kPw = kSel + ((sizeof(SelOut) + 15) & ~size_t(15));   // radix prefix (4 words)
  static constexpr size_t kNc = kPw + 16;                       // candidate count
  static constexpr size_t kHk = kNc + 16;                       // hash slot keys (far trade + 1; 0 = empty)
  static constexpr size_t kHist = kHk + size_t(kH) * 4;         // radix histogram
  static constexpr size_t kHb = kHist + (size_t(1) << B) * 4;   // slot block bytes (see block_flags)
  static constexpr size_t kBytes = (kHb + size_t(kH) * 4 + 15) & ~size_t(15);
  static_assert(kHk % 16 == 0 && kHist % 16 == 0 && kHb % 16 == 0, "16-byte aligned tables");
  char* base;
  __device__ __forceinline__ uint64_t* ck() const { return reinterpret_cast<uint64_t*>(base + kCk); }
  __device__ __forceinline__ uint64_t* ctb() const { return reinterpret_cast<uint64_t*>(base + kCtb); }
  __device__ __forceinline__ SelOut* sel() const { return reinterpret_cast<SelOut*>(base + kSel); }
  __device__ __forceinline__ uint32_t* pw() const { return reinterpret_cast<uint32_t*>(base + kPw); }
  __device__ __forceinline__ int32_t* ncand() const { return reinterpret_cast<int32_t*>(base + kNc); }
  __device__ __forceinline__ uint32_t* hk() const { return reinterpret_cast<uint32_t*>(base + kHk); }
  __device__ __forceinline__ uint32_t* hist() const { return reinterpret_cast<uint32_t*>(base + kHist); }
  __device__ __forceinline__ uint32_t* hb() const { return reinterpret_cast<uint32_t*>(base + kHb); }
};

// A slot's block word holds one byte per edge of the 2x2 block matrix
// (byte 2 rho + gamma: the trade's node rho adjacent to the far node
// 2s + gamma): 0 absent, 1 present, 3 present and moved by the trade.
// Plain byte stores fill it (the entries of one slot write different bytes,
// or equal values), so it needs no atomics.  block_flags turns it into the
// flag layout of the shared-memory path: presence bits 0..3, flips 4..7.
__device__ __forceinline__ uint32_t compact_bytes(uint32_t x) {   // x: bytes 0 or 1
  return (x | (x >> 7) | (x >> 14) | (x >> 21)) & 15u;
}
__device__ __forceinline__ uint32_t block_flags(uint32_t w) {
  return compact_bytes(w & 0x01010101u) | (compact_bytes((w >> 1) & 0x01010101u) << 4);
}
__device__ __forceinline__ void block_mark(uint32_t* hb, uint32_t slot, int q, uint8_t v) {
  reinterpret_cast<uint8_t*>(hb + slot)[q] = v;
}

// Trade t (nodes at t2u, t2u+1) depends on the earlier trade s through a
// block of two or more edges (flags f: bit 2 rho + gamma, t's node rho
// adjacent to s's node 2s + gamma): replay s's decisions on the block from
// its published threshold and return whether t's other node is adjacent to
// the s-node that the row-r entry of column colb ends on when t acts (a
// common neighbour).  Kept out of line: the path is rare, and inlined into
// every unrolled entry it would copy Philox many times over.
__device__ __noinline__ int replay_other(const uint64_t* thr_key, const uint64_t* thr_tb, KeyCtx kc, uint32_t t2u,
                                         uint32_t s, uint32_t f, int r, int colb) {
  const int u0 = f & 1, u1 = (f >> 1) & 1, v0 = (f >> 2) & 1, v1 = (f >> 3) & 1;
  const int bits[2][2] = {{u0, u1}, {v0, v1}};
  const int cnt_row[2] = {u0 + u1, v0 + v1};
  int m1[2][2] = {{0, 0}, {0, 0}};
  int col_now = colb;
  const uint64_t tk = __ldcg(thr_key + s), tt = __ldcg(thr_tb + s);
  for (int rho = 0; rho < 2; ++rho)
    for (int gam = 0; gam < 2; ++gam) {
      if (!bits[rho][gam]) continue;
      int g2 = gam;
      if (cnt_row[rho] == 1) {
        const uint32_t x = t2u + rho, yb = 2u * s + gam;
        const uint32_t lo = min(x, yb), hi = max(x, yb);
        const uint64_t k = side_key(kc, lo, hi, (lo >> 1) == s);
        g2 = at_or_below(k, tie_break(lo, hi), tk, tt) ? 0 : 1;
      }
      m1[rho][g2] = 1;
      if (rho == r && gam == colb) col_now = g2;
    }
  return m1[1 - r][col_now];
}

// Word d of an element's 128-bit order (key, lo, hi): key high, key low, lo, hi.
__device__ __forceinline__ uint32_t sel_word(int d, uint64_t key, uint32_t lo, uint32_t hi) {
  return d == 0 ? static_cast<uint32_t>(key >> 32) : d == 1 ? static_cast<uint32_t>(key) : d == 2 ? lo : hi;
}
// B bits of the 128-bit order starting q bits below its top.
__device__ __forceinline__ uint32_t sel_digit(int q, int B, uint64_t key, uint32_t lo, uint32_t hi) {
  const int w = q >> 5, off = q & 31;
  const uint64_t x = (static_cast<uint64_t>(sel_word(w, key, lo, hi)) << 32) |
                     (w < 3 ? sel_word(w + 1, key, lo, hi) : 0u);
  return static_cast<uint32_t>((x << off) >> (64 - B));
}
// Do the top q bits of the element's order equal those of the prefix pw?
__device__ __forceinline__ bool sel_match(int q, const uint32_t* pw, uint64_t key, uint32_t lo, uint32_t hi) {
  for (int d = 0; d < 4 && 32 * d < q; ++d) {
    const uint32_t a = sel_word(d, key, lo, hi), b = pw[d];
    const int bits = min(32, q - 32 * d);
    if (bits == 32 ? a != b : (a >> (32 - bits)) != (b >> (32 - bits))) return false;
  }
  return true;
}

// The step-start positions (lo, hi) of an entry's edge.
__device__ __forceinline__ void entry_lo_hi(uint32_t t2u, uint32_t m, uint32_t y, uint32_t* lo, uint32_t* hi) {
  const uint32_t x = t2u + ((m & kMR) ? 1u : 0u);
  *lo = min(x, y);
  *hi = max(x, y);
}

template <class Team, int J, int B, bool kKeepKey, bool kOneSeed = false, class Ws>
__device__ void phase_a_reg(Team& tm, const StepCtx& c, int64_t t, const Ws& w) {
  static_assert(Team::N <= 2048 && Team::N * J < (1 << 20), "reduction fields: 20-bit count, 12-bit flags");
  constexpr int NB = 1 << B;
  const TradeRows tr = trade_rows(c, t);
  const KeyCtx kc = key_ctx(c, t);
  const int du = tr.du, L = tr.du + tr.dv;
  // the new rows' offsets, loaded now so their two dependent loads overlap
  // the trade's work
  const int64_t ou = c.rp_next[__ldg(c.M + 2 * t)];
  const int64_t ov = tr.single ? 0 : c.rp_next[__ldg(c.M + 2 * t + 1)];
  // at least 4 hash slots per entry, and about one first-digit bin per entry
  const int lgH = max(5, 34 - __clz(max(L, 2) - 1));   // next power of two >= 4 L
  const int H = 1 << lgH;
  const int B0 = min(B, max(5, 32 - __clz(max(L - 1, 1))));
  const int NB0 = 1 << B0;
  const uint32_t t32 = static_cast<uint32_t>(t), T32 = static_cast<uint32_t>(c.T);
  const uint32_t t2u = 2u * t32;
  {
    // clear the tables in 16-byte stores (H and NB0 are powers of two >= 32;
    // the layout keeps every table 16-byte aligned)
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    uint4* hk4 = reinterpret_cast<uint4*>(w.hk());
    uint4* hb4 = reinterpret_cast<uint4*>(w.hb());
    uint4* hs4 = reinterpret_cast<uint4*>(w.hist());
    for (int i = tm.rank; i < (H >> 2); i += Team::N) {
      hk4[i] = z;
      hb4[i] = z;
    }
    for (int i = tm.rank; i < (NB0 >> 2); i += Team::N) hs4[i] = z;
  }
  if (tm.rank == 0) *w.ncand() = 0;
  tm.sync();
  // entries into the hash: presence bit (row, column) in the far trade's slot
  uint32_t y[J], mt[J], kt[J], kl[kKeepKey ? J : 1];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int i = tm.rank + j * Team::N;
    y[j] = 0;
    mt[j] = 0;
    kt[j] = 0;
    if (kKeepKey) kl[j] = 0;
    if (i < L) {
      const int32_t yy = __ldcg(c.col + tr.b0 + i);
      const uint32_t r = i >= du ? 1u : 0u;
      const uint32_t s = static_cast<uint32_t>(yy) >> 1;
      uint32_t m = kMValid | (r ? kMR : 0u) | ((yy & 1) ? kMCol : 0u);
      if (s == t32) m |= kMUV;
      else m |= hslot(s, lgH);
      y[j] = static_cast<uint32_t>(yy);
      mt[j] = m;
    }
  }
  // the hash (open addressing, far trade + 1 as key): every entry writes its
  // key into its home slot if that is empty (a plain store); after a barrier
  // it reads the slot back: its key (written by itself or by an entry of the
  // same far trade) places it; the few entries whose slot another key won
  // claim a further slot with a compare-and-swap.
  {
    uint32_t pend = 0;
#pragma unroll
    for (int j = 0; j < J; ++j)
      if ((mt[j] & kMValid) && !(mt[j] & kMUV)) pend |= 1u << j;
    // a warp or part of one repeats the plain round (its barriers are
    // cheap) until every entry is placed; a larger team runs one round, then
    // compare-and-swap
    // (the first round's slots are all empty or written in this round, so
    // its stores need no check).  An entry marks its edge in the slot's
    // block word as soon as its slot is final.
    constexpr bool kRounds = Team::N <= 32;
    bool first = true;
    for (;;) {
#pragma unroll
      for (int j = 0; j < J; ++j)
        if ((pend >> j) & 1u) {
          const uint32_t sl = mt[j] & kMSlot;
          if (first || w.hk()[sl] == 0u) w.hk()[sl] = (y[j] >> 1) + 1u;
        }
      first = false;
      tm.sync();
      bool more = false;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if ((pend >> j) & 1u) {
          const uint32_t sl = mt[j] & kMSlot;
          const uint32_t key = (y[j] >> 1) + 1u;
          const int q = 2 * ((mt[j] & kMR) ? 1 : 0) + ((mt[j] & kMCol) ? 1 : 0);
          if (w.hk()[sl] == key) {
            pend &= ~(1u << j);
            block_mark(w.hb(), sl, q, 1);
          } else if (kRounds) {
            mt[j] = (mt[j] & ~kMSlot) | ((sl + 1u) & static_cast<uint32_t>(H - 1));
            more = true;
          } else {   // lost the slot to another key: claim one further on
            const uint32_t sl2 = h_claim(w.hk(), static_cast<uint32_t>(H - 1), key, (sl + 1u) & (H - 1));
            mt[j] = (mt[j] & ~kMSlot) | sl2;
            block_mark(w.hb(), sl2, q, 1);
          }
        }
      if (!kRounds || !tm.any(more)) break;
    }
  }
  tm.sync();
  // block analysis, keys, histogram of the first radix digit
  bool defer = false, has_dependents = false, any_multi = false;
  int cnt_a = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    uint32_t m = mt[j];
    if (!(m & kMValid) || (m & kMUV)) continue;
    const int r = (m & kMR) ? 1 : 0;
    const uint32_t colb = (m & kMCol) ? 1u : 0u;
    const uint32_t s = y[j] >> 1;
    const uint32_t f = block_flags(w.hb()[m & kMSlot]) & 15u;
    int other = 0;   // the other row is adjacent to this neighbour when t acts
    if (f & (f - 1u)) {
      // a block of two or more edges: common neighbours and dependencies
      m |= kMMulti;
      any_multi = true;
      const int u0 = f & 1, u1 = (f >> 1) & 1, v0 = (f >> 2) & 1, v1 = (f >> 3) & 1;
      const int cu = u0 + u1, cv = v0 + v1;
      if (!tr.single && s > t32 && s < T32 && (u0 + v0 == 1 || u1 + v1 == 1)) has_dependents = true;
      int col_now = static_cast<int>(colb);
      other = r ? (col_now ? u1 : u0) : (col_now ? v1 : v0);
      if (!tr.single && s < t32 && (cu == 1 || cv == 1)) {
        // unpublished: a parallel pass leaves the trade to a later pass,
        // an in-order pass waits
        if (ld_acquire(c.done + s) != c.stamp &&
            !(c.wait && wait_published(c.done + s, c.err, c.stamp, c.wait_ns))) {
          defer = true;
          mt[j] = m;
          continue;
        }
        other = replay_other(c.thr_key, c.thr_tb, kc, t2u, s, f, r, static_cast<int>(colb));
      }
    }
    // both trades' keys of this edge (step-start positions)
    const uint32_t x = t2u + r, yb = y[j];
    const uint32_t lo = min(x, yb), hi = max(x, yb);
    const EdgeKeys ek = edge_keys<kOneSeed>(c, kc, lo, hi);
    const bool lo_mine = (lo >> 1) == t32;
    const uint64_t own = lo_mine ? ek.lo_side : ek.hi_side;
    const uint64_t far = lo_mine ? ek.hi_side : ek.lo_side;
    kt[j] = static_cast<uint32_t>(own >> 32);
    if (kKeepKey) kl[j] = static_cast<uint32_t>(own);
    m |= static_cast<uint32_t>(far >> (64 - kFarBits)) << kMFarShift;
    if (!other && !tr.single) {
      m |= kMInD;
      cnt_a += (r == 0);
      atomicAdd(&w.hist()[kt[j] >> (32 - B0)], 1u);
    }
    mt[j] = m;
  }
  // one reduction: |A_{u-v}| (bits 0..19) and, in 12-bit fields that hold a
  // count over up to 1024 members, the members that saw a deferral, a later
  // dependent trade, a multi-edge block
  const int64_t tot = tm.sum(static_cast<int64_t>(cnt_a) | (static_cast<int64_t>(defer) << 20) |
                             (static_cast<int64_t>(has_dependents) << 32) | (static_cast<int64_t>(any_multi) << 44));
  if ((tot >> 20) & 0xfff) {
    if (tm.rank == 0) defer_trade(c, t, L);
    tm.sync();
    return;
  }
  const int a = static_cast<int>(tot & 0xfffff);
  const bool publish_fence = ((tot >> 32) & 0xfff) != 0;
  const bool multi_any = ((tot >> 44) & 0xfff) != 0;
  const bool no_thr = tr.single || a == 0;   // u keeps nothing of D
  uint64_t tk = 0, tt = 0;
  if (!no_thr) {
    // the bin of the first digit (top B0 key bits) that holds the a-th smallest element
    constexpr int BPM = (NB + Team::N - 1) / Team::N;
    {
      const int bpm0 = (NB0 + Team::N - 1) / Team::N;
      const int b0 = tm.rank * bpm0;
      int local = 0;
#pragma unroll
      for (int q = 0; q < BPM; ++q)
        if (q < bpm0 && b0 + q < NB0) local += static_cast<int>(w.hist()[b0 + q]);
      int run = static_cast<int>(tm.exscan(local));
#pragma unroll
      for (int q = 0; q < BPM; ++q) {
        const int b = b0 + q;
        if (q < bpm0 && b < NB0) {
          const int hc = static_cast<int>(w.hist()[b]);
          if (run < a && a <= run + hc) {
            w.sel()->bin = b;
            w.sel()->below = run;
            w.sel()->cnt = hc;
          }
          run += hc;
        }
      }
    }
    tm.sync();
    int qbits = B0;             // top bits of the order fixed so far
    int kk = a - w.sel()->below;  // rank sought among the elements sharing them
    int cnt = w.sel()->cnt;
    if (tm.rank == 0) {
      w.pw()[0] = static_cast<uint32_t>(w.sel()->bin) << (32 - B0);
      w.pw()[1] = w.pw()[2] = w.pw()[3] = 0u;
    }
    tm.sync();
    // more elements share the prefix than the candidate list holds (or the
    // list is disabled): further B-bit digits of (key, lo, hi)
    while (cnt > c.cand_max) {
      for (int i = tm.rank; i < NB; i += Team::N) w.hist()[i] = 0u;
      tm.sync();
#pragma unroll
      for (int j = 0; j < J; ++j) {
        if (!(mt[j] & kMInD)) continue;
        uint32_t lo, hi;
        entry_lo_hi(t2u, mt[j], y[j], &lo, &hi);
        const uint64_t key = kKeepKey ? ((static_cast<uint64_t>(kt[j]) << 32) | kl[j]) : own_key(kc, t, lo, hi);
        if (sel_match(qbits, w.pw(), key, lo, hi)) atomicAdd(&w.hist()[sel_digit(qbits, B, key, lo, hi)], 1u);
      }
      tm.sync();
      {
        const int b0 = tm.rank * BPM;
        int local = 0;
#pragma unroll
        for (int q = 0; q < BPM; ++q)
          if (b0 + q < NB) local += static_cast<int>(w.hist()[b0 + q]);
        int run = static_cast<int>(tm.exscan(local));
#pragma unroll
        for (int q = 0; q < BPM; ++q) {
          const int b = b0 + q;
          if (b < NB) {
            const int hc = static_cast<int>(w.hist()[b]);
            if (run < kk && kk <= run + hc) {
              w.sel()->bin = b;
              w.sel()->below = run;
              w.sel()->cnt = hc;
            }
            run += hc;
          }
        }
      }
      tm.sync();
      const uint32_t dig = static_cast<uint32_t>(w.sel()->bin);
      kk -= w.sel()->below;
      cnt = w.sel()->cnt;
      tm.sync();
      if (tm.rank == 0) {   // append the digit to the prefix (it may straddle two words)
        const int wd = qbits >> 5, off = qbits & 31;
        const uint64_t d64 = static_cast<uint64_t>(dig) << (64 - B - off);
        w.pw()[wd] |= static_cast<uint32_t>(d64 >> 32);
        if (wd < 3) w.pw()[wd + 1] |= static_cast<uint32_t>(d64);
      }
      qbits += B;
      tm.sync();
    }
    // rank the few elements that share the prefix by their full order
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!(mt[j] & kMInD)) continue;
      if (qbits == B0 && (kt[j] >> (32 - B0)) != (w.pw()[0] >> (32 - B0))) continue;
      uint32_t lo, hi;
      entry_lo_hi(t2u, mt[j], y[j], &lo, &hi);
      const uint64_t key = kKeepKey ? ((static_cast<uint64_t>(kt[j]) << 32) | kl[j]) : own_key(kc, t, lo, hi);
      if (qbits > B0 && !sel_match(qbits, w.pw(), key, lo, hi)) continue;
      if (cnt == 1) {
        w.sel()->key = key;
        w.sel()->tb = tie_break(lo, hi);
      } else {
        const int q = atomicAdd(w.ncand(), 1);
        w.ck()[q] = key;
        w.ctb()[q] = tie_break(lo, hi);
      }
    }
    tm.sync();
    if (cnt > 1) {
      for (int q = tm.rank; q < cnt; q += Team::N) {
        int rk = 0;
        for (int p = 0; p < cnt; ++p) rk += (w.ck()[p] < w.ck()[q] || (w.ck()[p] == w.ck()[q] && w.ctb()[p] < w.ctb()[q]));
        if (rk == kk - 1) {
          w.sel()->key = w.ck()[q];
          w.sel()->tb = w.ctb()[q];
        }
      }
      tm.sync();
    }
    tk = w.sel()->key;
    tt = w.sel()->tb;
  }
  // own decisions: u keeps the elements at or below the threshold
  const uint32_t tk32 = static_cast<uint32_t>(tk >> 32);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const uint32_t m = mt[j];
    if (!(m & kMInD)) continue;
    const int r = (m & kMR) ? 1 : 0;
    bool low;
    if (no_thr) {
      low = false;
    } else if (kt[j] != tk32) {
      low = kt[j] < tk32;
    } else {
      uint32_t lo, hi;
      entry_lo_hi(t2u, m, y[j], &lo, &hi);
      const uint64_t key = kKeepKey ? ((static_cast<uint64_t>(kt[j]) << 32) | kl[j]) : own_key(kc, t, lo, hi);
      low = at_or_below(key, tie_break(lo, hi), tk, tt);
    }
    if ((low ? 0 : 1) != r) {
      mt[j] = m | kMFlip;
      if (m & kMMulti) block_mark(w.hb(), m & kMSlot, 2 * r + ((m & kMCol) ? 1 : 0), 3);
    }
  }
  if (multi_any) tm.sync();
  // placement: each entry goes into the new row of its node after the trade
  // (u's or v's row of step g+1) at a slot given by a scan over the team
  int n0 = 0, n1 = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const uint32_t m = mt[j];
    if (!(m & kMValid)) continue;
    const int side = ((m & kMR) ? 1 : 0) ^ ((m & kMFlip) ? 1 : 0);
    n0 += side == 0;
    n1 += side;
  }
  const int64_t pre = tm.exscan(static_cast<int64_t>(n0) | (static_cast<int64_t>(n1) << 32));
  int s0 = static_cast<int>(pre & 0xffffffff), s1 = static_cast<int>(pre >> 32);
  if (tm.rank == Team::N - 1 && (s0 + n0 != du || s1 + n1 != tr.dv)) latch(c.err, kErrRowLength);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const uint32_t m = mt[j];
    if (!(m & kMValid)) continue;
    const int r = (m & kMR) ? 1 : 0;
    const int f = (m & kMFlip) ? 1 : 0;
    // will the far trade decide this edge?  (A single-edge block: yes,
    // unless the far node is the untraded one of an odd n, trade index T.)
    int in_far = 0;
    if (!(m & kMUV)) {
      const uint32_t s = y[j] >> 1;
      if (!(m & kMMulti)) {
        in_far = s < T32;
      } else if (tr.single || s < t32) {
        const uint32_t fl = block_flags(w.hb()[m & kMSlot]);
        in_far = __popc(r ? (fl & 12u) : (fl & 3u)) == 1;   // trade s acted before t: initial block
      } else if (s < T32) {   // block after t's own decisions: presence bits 0..3, flips 4..7
        const uint32_t fl = block_flags(w.hb()[m & kMSlot]);
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
    const int side = r ^ f;
    const int k = side ? s1++ : s0++;
    if (k >= (side ? tr.dv : du)) continue;   // counts checked above: never write outside the row
    const int64_t slot = (side ? ov : ou) + k;
    c.ph[slot] = static_cast<int32_t>(y[j]);
    c.fb[slot] = static_cast<uint16_t>(f | (in_far ? (((m >> kMFarShift) << 1) | kFbInFar) : 0u));
  }
  if (tm.rank == 0 && !tr.single) {
    c.thr_key[t] = tk;
    c.thr_tb[t] = tt;
    c.thr_top[t] = static_cast<uint8_t>(tk >> 56);
    if (publish_fence && !c.hold_publish) {
      __threadfence();
      st_release(c.done + t, c.stamp);
    } else if (!publish_fence) {
      c.done[t] = kComplete;   // a deferred trade done in a retry pass leaves the deferred list
    }
  }
  tm.sync();
}

// Phase A of small trades, one warp per trade (L <= 32 J): eight independent
// warps per CTA, each with its own workspace; no CTA barriers.
constexpr int kWarpJ = 4;                       // entries per lane: trades up to 128 entries
constexpr int kWarpB = 7;                       // first radix digit: 128 bins
constexpr int kWarpWarps = 8;                   // warps per CTA
using WarpWs = RegWs<32 * kWarpJ, kWarpB>;

// The smallest trades (L <= W J, W = 8 or 16) on teams of W lanes: 32 / W
// trades per warp, so the per-trade work (clearing the tables, scans,
// reductions, the threshold search) takes one warp instruction for all of
// them.
template <int W>
struct LaneCfg {
  static constexpr int B = W == 8 ? 5 : 6;   // ~1 first-digit bin per entry
  using Ws = RegWs<W * kWarpJ, B>;
  static constexpr int kTeams = 32 * kWarpWarps / W;   // teams per CTA
  static constexpr size_t kSmem = Ws::kBytes * kTeams;
};
template <int W>
__global__ void __launch_bounds__(32 * kWarpWarps, 4) k_phase_a_lanes(StepCtx c, const int32_t* __restrict__ lists,
                                                                   const int64_t* __restrict__ ctr, int cls) {
  using Cfg = LaneCfg<W>;
  extern __shared__ __align__(16) char lsm[];
  const int id = threadIdx.x / W;
  const typename Cfg::Ws w{lsm + Cfg::Ws::kBytes * id};
  LaneTeam<W> tm;
  const ClassList cl = class_list(lists, ctr, cls);
  const int64_t step = static_cast<int64_t>(gridDim.x) * Cfg::kTeams;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * Cfg::kTeams + id; q < cl.len; q += step)
    phase_a_reg<LaneTeam<W>, kWarpJ, Cfg::B, true>(tm, c, cl.list[q], w);
}

__global__ void __launch_bounds__(32 * kWarpWarps, 4) k_phase_a_warp(StepCtx c, const int32_t* __restrict__ lists,
                                                                  const int64_t* __restrict__ ctr, int cls) {
  extern __shared__ __align__(16) char wsm[];
  const int wid = threadIdx.x >> 5;
  const WarpWs w{wsm + WarpWs::kBytes * wid};
  WarpTeam tm;
  const ClassList cl = class_list(lists, ctr, cls);
  const int64_t step = static_cast<int64_t>(gridDim.x) * kWarpWarps;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * kWarpWarps + wid; q < cl.len; q += step)
    phase_a_reg<WarpTeam, kWarpJ, kWarpB, true>(tm, c, cl.list[q], w);
}

// Phase A of larger trades: a CTA of CT threads holds CT / NT teams of NT
// threads (named barriers), each running one trade at a time with kTeamJ
// entries per thread in registers (L <= NT kTeamJ).
constexpr int kTeamJ = 4;
template <int NT>
struct TeamCfg {
  static constexpr int B = NT == 64 ? 8 : NT == 128 ? 9 : NT == 256 ? 10 : NT == 512 ? 11 : 12;   // ~1 bin per entry
  using Ws = RegWs<NT * kTeamJ, B>;
  static constexpr int kMax = NT * kTeamJ;
};
template <int CT, int NT, bool kOneSeed>
__global__ void __launch_bounds__(CT, CT == 256 ? 4 : 1) k_phase_a_team(StepCtx c, const int32_t* __restrict__ lists,
                                                                      const int64_t* __restrict__ ctr, int cls) {
  constexpr int kTeams = CT / NT;
  using Ws = typename TeamCfg<NT>::Ws;
  extern __shared__ __align__(16) char tsm[];
  __shared__ int64_t red[kTeams * SubTeam<NT>::kRedSlots];
  const int id = threadIdx.x / NT;
  SubTeam<NT> tm(red + id * SubTeam<NT>::kRedSlots, id);
  const Ws w{tsm + Ws::kBytes * id};
  const ClassList cl = class_list(lists, ctr, cls);
  const int64_t step = static_cast<int64_t>(gridDim.x) * kTeams;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * kTeams + id; q < cl.len; q += step)
    phase_a_reg<SubTeam<NT>, kTeamJ, TeamCfg<NT>::B, false, kOneSeed>(tm, c, cl.list[q], w);
}
template <int CT, int NT>
constexpr size_t team_smem() {
  return TeamCfg<NT>::Ws::kBytes * (CT / NT);
}

// ---------------------------------------------------------- classification
//
// Every trade falls into one of kClasses size classes (by L = deg u + deg v
// against ascending thresholds), each run by its own team size.  The class
// lists are one stable counting sort: counts per class and 2048-trade chunk,
// one exclusive scan of those counts in class-major order (so each class's
// list follows the previous class's), then every chunk places its trades,
// in index order within each class.

constexpr int kClassThreads = 256;
constexpr int kClassPer = 8;
constexpr int kClassChunk = kClassThreads * kClassPer;   // trades per chunk

struct ClassTh {
  int th[kClasses - 1];   // class k holds th[k-1] < L <= th[k] (th[-1] = -1, th[kClasses-1] = inf)
};
__device__ __forceinline__ int trade_class(const ClassTh& th, int L) {
  int k = 0;
#pragma unroll
  for (int i = 0; i < kClasses - 1; ++i) k += L > th.th[i];
  return k;
}

// The first classification of a step also adds up every class's directed
// entries (L summed) into ctr[kCtrFirstEnt + k], for the stats.
__global__ void __launch_bounds__(kClassThreads) k_class_count(StepCtx c, int64_t ntasks, ClassTh th,
                                                               int64_t nchunks, int only_deferred,
                                                               int32_t* __restrict__ counts,
                                                               int64_t* __restrict__ ctr) {
  __shared__ int wc[kClassThreads / 32][kClasses];
  __shared__ unsigned long long we[kClasses];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < kClasses) we[threadIdx.x] = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    int mine[kClasses] = {};
    unsigned ent[kClasses] = {};
    for (int j = 0; j < kClassPer; ++j) {
      const int64_t t = ch * kClassChunk + j * kClassThreads + threadIdx.x;
      int k = -1, L = 0;
      if (t < ntasks && (!only_deferred || __ldcg(c.done + t) == kDeferred)) {
        const TradeRows tr = trade_rows(c, t);
        L = tr.du + tr.dv;
        k = trade_class(th, L);
      }
#pragma unroll
      for (int q = 0; q < kClasses; ++q) {
        mine[q] += __popc(__ballot_sync(kFull, k == q));
        ent[q] += k == q ? static_cast<unsigned>(L) : 0u;
      }
    }
    if (lane == 0)
      for (int q = 0; q < kClasses; ++q) wc[warp][q] = mine[q];
    if (!only_deferred) {
#pragma unroll
      for (int q = 0; q < kClasses; ++q) {
        const unsigned e = __reduce_add_sync(kFull, ent[q]);
        if (lane == 0 && e) atomicAdd(&we[q], static_cast<unsigned long long>(e));
      }
    }
    __syncthreads();
    if (threadIdx.x < kClasses) {
      int tot = 0;
      for (int w = 0; w < kClassThreads / 32; ++w) tot += wc[w][threadIdx.x];
      counts[threadIdx.x * nchunks + ch] = tot;
    }
    __syncthreads();
  }
  if (!only_deferred && threadIdx.x < kClasses && we[threadIdx.x])
    atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrFirstEnt + threadIdx.x), we[threadIdx.x]);
}

__global__ void __launch_bounds__(kClassThreads) k_class_place(StepCtx c, int64_t ntasks, ClassTh th,
                                                               int64_t nchunks, int only_deferred,
                                                               const int64_t* __restrict__ off,
                                                               int32_t* __restrict__ lists) {
  __shared__ int wc[kClassThreads / 32][kClasses];
  __shared__ int64_t base[kClasses];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    if (threadIdx.x < kClasses) base[threadIdx.x] = off[threadIdx.x * nchunks + ch];
    __syncthreads();
    for (int j = 0; j < kClassPer; ++j) {
      const int64_t t = ch * kClassChunk + j * kClassThreads + threadIdx.x;
      int k = -1;
      if (t < ntasks && (!only_deferred || __ldcg(c.done + t) == kDeferred)) {
        const TradeRows tr = trade_rows(c, t);
        k = trade_class(th, tr.du + tr.dv);
      }
      unsigned same = 0;
#pragma unroll
      for (int q = 0; q < kClasses; ++q) {
        const unsigned b = __ballot_sync(kFull, k == q);
        if (k == q) same = b;
        if (lane == 0) wc[warp][q] = __popc(b);
      }
      __syncthreads();
      if (k >= 0) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wc[w][k];
        lists[base[k] + before + __popc(same & below)] = static_cast<int32_t>(t);
      }
      __syncthreads();
      if (threadIdx.x < kClasses) {
        int tot = 0;
        for (int w = 0; w < kClassThreads / 32; ++w) tot += wc[w][threadIdx.x];
        base[threadIdx.x] += tot;
      }
      __syncthreads();
    }
  }
}

// Each class's first list entry and length into the counters (for the
// first classification of a step also into the stats' copy).
__global__ void k_class_bounds(const int64_t* __restrict__ off, int64_t nchunks, int first,
                               int64_t* __restrict__ ctr) {
  const int k = threadIdx.x;
  if (k < kClasses) {
    const int64_t len = off[(k + 1) * nchunks] - off[k * nchunks];
    ctr[kCtrClsStart + k] = off[k * nchunks];
    ctr[kCtrClsLen + k] = len;
    if (first) ctr[kCtrFirstLen + k] = len;
  }
}

// ------------------------------------------------------ rebuild: fix-up
//
// Phase A leaves every entry in its new row (step g+1 layout) as a
// placeholder: the far end's step-g position y, and a side word (bit 0 the
// own trade's flip, bits 1..kFarBits the top bits of the far trade's key for
// the edge, bit 12 set when the far trade decides the edge).  The fix-up
// replaces each placeholder by the step-(g+1) position of the far end: y
// itself, or the node of y's trade that the trade's threshold gives it.  One
// 8-byte record per far trade holds both of its nodes' new positions and its
// threshold's top 8 bits; the pass runs once per slice of far trades small
// enough for the records to stay in L2, each pass reading every placeholder
// and writing the entries of its slice.  Equal 8-bit prefixes (1 in 256)
// fetch the far threshold's longer prefix; a tie there too (1 in 2^kFarBits)
// needs the full key, hence the edge's own end at the start of the step: the
// node of the entry's row (found by a search of the chunk's row offsets)
// before the own flip.

constexpr int kFixThreads = 256;
constexpr int kFixPer = 8;                             // consecutive entries per thread
constexpr int kFixChunk = kFixThreads * kFixPer;       // entries per chunk

// Rows whose entries contain each chunk's first entry (one thread per row:
// every chunk start lies in exactly one non-empty row); the last entry holds
// the last row.
__global__ void k_chunk_rows(int64_t nrows, const int64_t* __restrict__ rp, int64_t nchunks,
                             int32_t* __restrict__ chunk_row) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows; p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = rp[p], b = rp[p + 1];
    for (int64_t ch = (a + kFixChunk - 1) / kFixChunk; ch < nchunks && ch * kFixChunk < b; ++ch)
      chunk_row[ch] = static_cast<int32_t>(p);
    if (p == nrows - 1) chunk_row[nchunks] = static_cast<int32_t>(p);
  }
}

// What the fix-up needs of a far trade s: the new positions of its two nodes
// and the top 8 bits of its threshold key.  Up to 2^28 positions it fits 8
// bytes (28 + 28 + 8 bits), else 16.
constexpr int64_t kNarrowPackMax = int64_t(1) << 28;

struct FarTrade {
  int32_t x, y;    // new positions of nodes 2s and 2s+1
  uint32_t top;    // threshold prefix (8 bits)
};

template <bool kNarrow>
__global__ void k_far_pack(StepCtx c, int64_t ntasks, void* __restrict__ pack) {
  for (int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; s < ntasks; s += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t x = static_cast<uint32_t>(c.M[2 * s]);
    const uint32_t y = 2 * s + 1 < c.n ? static_cast<uint32_t>(c.M[2 * s + 1]) : 0u;
    const uint32_t top = 2 * s + 1 < c.n ? c.thr_top[s] : 0u;
    if constexpr (kNarrow) {
      static_cast<uint64_t*>(pack)[s] = uint64_t(x) | (uint64_t(y) << 28) | (uint64_t(top) << 56);
    } else {
      static_cast<int4*>(pack)[s] = make_int4(static_cast<int32_t>(x), static_cast<int32_t>(y),
                                              static_cast<int32_t>(top), 0);
    }
  }
}

// The record as loaded: 8 bytes, or 16 for the wide layout.
template <bool kNarrow>
struct FarRaw {
  uint64_t v;
};
template <>
struct FarRaw<false> {
  int4 v;
};
template <bool kNarrow>
__device__ __forceinline__ FarRaw<kNarrow> far_raw(const void* pack, uint32_t s) {
  if constexpr (kNarrow) return {__ldg(static_cast<const unsigned long long*>(pack) + s)};
  else return {__ldg(static_cast<const int4*>(pack) + s)};
}
template <bool kNarrow>
__device__ __forceinline__ FarTrade far_decode(const FarRaw<kNarrow>& r) {
  if constexpr (kNarrow) {
    return {static_cast<int32_t>(r.v & 0x0FFFFFFFu), static_cast<int32_t>((r.v >> 28) & 0x0FFFFFFFu),
            static_cast<uint32_t>(r.v >> 56)};
  } else {
    return {r.v.x, r.v.y, static_cast<uint32_t>(r.v.z)};
  }
}

template <bool kNarrow>
__device__ __forceinline__ FarTrade far_trade(const void* pack, uint32_t s) {
  if constexpr (kNarrow) {
    const uint64_t v = __ldg(static_cast<const unsigned long long*>(pack) + s);
    return {static_cast<int32_t>(v & 0x0FFFFFFFu), static_cast<int32_t>((v >> 28) & 0x0FFFFFFFu),
            static_cast<uint32_t>(v >> 56)};
  } else {
    const int4 v = __ldg(static_cast<const int4*>(pack) + s);
    return {v.x, v.y, static_cast<uint32_t>(v.z)};
  }
}

// Row (step g+1 position) holding entry e of chunk ch.
__device__ __forceinline__ int64_t fix_row(const StepCtx& c, const int32_t* chunk_row, int64_t ch, int64_t e) {
  int64_t lo = chunk_row[ch], hi = chunk_row[ch + 1];
  while (lo < hi) {   // last row whose first entry is <= e
    const int64_t mid = (lo + hi + 1) >> 1;
    if (c.rp_next[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kFixQueue = 2 * kFixChunk;    // prefix ties a CTA defers before resolving them together

// The kFixPer placeholders and side words of a thread starting at entry base
// (entries at or past nnz read as 0xFFFFFFFF).
template <bool kStream>
__device__ __forceinline__ void fix_load(const int32_t* ph, const uint16_t* fb, int64_t base, int64_t nnz,
                                         uint32_t* pv, uint32_t* bv) {
  if (base + kFixPer <= nnz) {   // 32 B and 16 B, aligned: chunks start at multiples of 2048 entries
    const uint4* p4 = reinterpret_cast<const uint4*>(ph + base);
    const uint4 a0 = kStream ? __ldcs(p4) : __ldcg(p4);
    const uint4 a1 = kStream ? __ldcs(p4 + 1) : __ldcg(p4 + 1);
    pv[0] = a0.x; pv[1] = a0.y; pv[2] = a0.z; pv[3] = a0.w;
    pv[4] = a1.x; pv[5] = a1.y; pv[6] = a1.z; pv[7] = a1.w;
    const uint4 b = __ldcs(reinterpret_cast<const uint4*>(fb + base));
    bv[0] = b.x; bv[1] = b.y; bv[2] = b.z; bv[3] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < kFixPer / 2; ++j) bv[j] = 0;
#pragma unroll
    for (int j = 0; j < kFixPer; ++j) {
      const bool in = base + j < nnz;
      pv[j] = in ? static_cast<uint32_t>(ph[base + j]) : 0xFFFFFFFFu;
      if (in) bv[j >> 1] |= static_cast<uint32_t>(fb[base + j]) << (16 * (j & 1));
    }
  }
}

// The new position of entry e's far end when its 8-bit key prefix equals
// the far threshold's: the threshold's longer prefix, and on a tie there too
// the full key of the edge (its own end at the start of the step is the
// node of the entry's row before the own flip).
template <bool kNarrow>
__device__ uint32_t fix_tie(const StepCtx& c, const void* pack, const int32_t* chunk_row, int64_t e, uint32_t y,
                            uint32_t b) {
  const uint32_t s = y >> 1;
  const FarTrade ft = far_trade<kNarrow>(pack, s);
  const uint32_t fp = (b >> 1) & ((1u << kFarBits) - 1u);
  const uint32_t tp = static_cast<uint32_t>(__ldcg(c.thr_key + s) >> (64 - kFarBits));
  bool low;
  if (fp != tp) {
    low = fp < tp;
  } else {
    const uint32_t xr = static_cast<uint32_t>(c.Minv[fix_row(c, chunk_row, e / kFixChunk, e)]) ^ (b & 1u);
    low = far_keeps_low(c, key_ctx(c, s), s, min(xr, y), max(xr, y));
  }
  return static_cast<uint32_t>(low ? ft.x : ft.y);
}

// One pass over far trades [s_lo, s_hi).  A pass other than the last writes
// the new positions of its entries into the placeholders (marked kPhDone);
// the last one writes every entry's new position to `out` in full vectors.
// Entries whose 8-bit prefix ties wait in a per-CTA queue and are resolved
// together, so that their extra loads hold up no warp.
template <bool kNarrow, bool kLast>
__global__ void __launch_bounds__(kFixThreads, 4) k_fixup(StepCtx c, int64_t nnz, uint32_t s_lo, uint32_t s_hi,
                                                       int32_t* __restrict__ ph, const uint16_t* __restrict__ fb,
                                                       int32_t* __restrict__ out, const void* __restrict__ pack,
                                                       const int32_t* __restrict__ chunk_row) {
  __shared__ int64_t qe[kFixQueue];
  __shared__ int qn;
  if (threadIdx.x == 0) qn = 0;
  __syncthreads();
  auto flush = [&]() {
    const int k = qn;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const int64_t e = qe[i];
      const uint32_t y = static_cast<uint32_t>(ph[e]);
      const uint32_t v = fix_tie<kNarrow>(c, pack, chunk_row, e, y, fb[e]);
      if (kLast) out[e] = static_cast<int32_t>(v);
      else ph[e] = static_cast<int32_t>(v | kPhDone);
    }
    __syncthreads();
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
  };
  const int64_t nchunks = (nnz + kFixChunk - 1) / kFixChunk;
  const int64_t tofs = static_cast<int64_t>(threadIdx.x) * kFixPer;
  uint32_t pv[kFixPer], bv[kFixPer / 2];
  int64_t ch = blockIdx.x;
  if (ch < nchunks) fix_load<kLast>(ph, fb, ch * kFixChunk + tofs, nnz, pv, bv);
  for (; ch < nchunks; ch += gridDim.x) {
    const int64_t base = ch * kFixChunk + tofs;
    // the next chunk's loads go out before this chunk's gathers
    uint32_t pn[kFixPer], bn[kFixPer / 2];
    const int64_t nxt = ch + gridDim.x;
    if (nxt < nchunks) fix_load<kLast>(ph, fb, nxt * kFixChunk + tofs, nnz, pn, bn);
    // first every gather of the thread's entries in this slice, then the decisions
    uint32_t res[kFixPer];
    FarRaw<kNarrow> ftv[kFixPer];
    uint32_t todo = 0;   // bit j: entry j is this pass's
#pragma unroll
    for (int j = 0; j < kFixPer; ++j) {
      const uint32_t p = pv[j];
      res[j] = (p & kPhDone) && p != 0xFFFFFFFFu ? (p & ~kPhDone) : 0u;   // an earlier pass resolved it
      const uint32_t s = p >> 1;
      const bool mine = !(p & kPhDone) && s >= s_lo && s < s_hi && p < static_cast<uint32_t>(c.n);
      if (!(p & kPhDone) && p >= static_cast<uint32_t>(c.n)) latch(c.err, kErrRowLength);   // a slot phase A did not fill
      if (mine) ftv[j] = far_raw<kNarrow>(pack, s);
      todo |= static_cast<uint32_t>(mine) << j;
    }
#pragma unroll
    for (int j = 0; j < kFixPer; ++j) {
      if (!((todo >> j) & 1u)) continue;
      const uint32_t y = pv[j];
      const FarTrade ft = far_decode<kNarrow>(ftv[j]);
      const uint32_t b = (bv[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      int side = static_cast<int>(y & 1u);
      if (b & kFbInFar) {   // the far trade decides: key prefixes first
        const uint32_t f8 = ((b >> 1) & ((1u << kFarBits) - 1u)) >> (kFarBits - 8);
        if (f8 == ft.top) {   // 1 in 256: resolved with the queue
          qe[atomicAdd(&qn, 1)] = base + j;
          continue;
        }
        side = f8 < ft.top ? 0 : 1;
      }
      res[j] = static_cast<uint32_t>(side ? ft.y : ft.x);
      if (!kLast) ph[base + j] = static_cast<int32_t>(res[j] | kPhDone);
    }
    if (kLast) {
      if (base + kFixPer <= nnz) {
        uint4* o4 = reinterpret_cast<uint4*>(out + base);
        __stcs(o4, make_uint4(res[0], res[1], res[2], res[3]));
        __stcs(o4 + 1, make_uint4(res[4], res[5], res[6], res[7]));
      } else {
#pragma unroll
        for (int j = 0; j < kFixPer; ++j)
          if (base + j < nnz) out[base + j] = static_cast<int32_t>(res[j]);
      }
    }
    __syncthreads();   // queued entries (and, on the last pass, their vector stores) are in place
    if (qn > kFixQueue - kFixChunk) flush();   // room for a whole chunk more
#pragma unroll
    for (int j = 0; j < kFixPer; ++j) pv[j] = pn[j];
#pragma unroll
    for (int j = 0; j < kFixPer / 2; ++j) bv[j] = bn[j];
  }
  __syncthreads();
  flush();
}

// ---------------------------------------------------------------- team paths

template <int NT, bool kOneSeed>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) k_phase_a_block(StepCtx c, const int32_t* __restrict__ lists,
                                                      const int64_t* __restrict__ ctr, int cls, int smem_max,
                                                      char* gws, size_t slice, int stage_cap) {
  // dynamic shared memory: the workspace, then the staging buffer of a
  // trade's entries (stage_cap + 8 int32, 16-byte aligned)
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ SelOut sel;
  __shared__ uint64_t mbar;
  BlockTeam<NT> tm(red);
  const ClassList cl = class_list(lists, ctr, cls);
  const int32_t* list = cl.list;
  const int64_t len = cl.len;
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
      const bool late = !mbar_wait(&mbar, parity, c.wait_ns);
      parity ^= 1;
      if (__syncthreads_or(late)) {
        failed = true;
        break;
      }
      ys = stage + stage_off(tr.b0);
    }
    phase_a<BlockTeam<NT>, kOneSeed>(tm, c, t, carve_a(base, L), &sel, ys, sn);
  }
  if (failed) {   // a copy did not complete in time: report, let it land, leave
    if (threadIdx.x == 0) latch(c.err, kErrStage);
    mbar_wait(&mbar, parity ^ 1, c.wait_ns);
  }
}

// The trades still deferred after the retry passes, in index order, found
// by scanning every trade's done flag.  CTAs claim chunks of
// trade indices in increasing order and run the deferred trades of a chunk one
// after another; a trade waits for an unpublished dependency instead of
// deferring.  A dependency s < t is either complete (first pass) or deferred
// too, and then it sits in an earlier chunk or earlier in the same chunk:
// claimed before t by a CTA that is already running.  By induction on the
// index, the smallest unfinished claimed trade waits for nothing, so every
// wait ends whatever the residency of the grid.
// It runs when the deferred trades did not fit the sorted list (skip = the
// list's flag, nonzero when k_phase_a_list runs them instead).
template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) k_phase_a_inorder(StepCtx c, int64_t ntasks, int64_t chunk,
                                                        unsigned long long* claim, int smem_max, char* gws,
                                                        size_t slice, const int64_t* skip) {
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ SelOut sel;
  __shared__ int64_t first;
  __shared__ int32_t found[NT];
  __shared__ int nfound;
  if (*reinterpret_cast<const volatile int64_t*>(skip)) return;
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

// The retry passes and, when the list could be sorted, the in-order pass,
// over explicit lists of deferred trades.  CTAs claim positions one at a
// time (list[p], or list[-1 - p] when from_back, for p < *count) and run the
// trades of L = deg u + deg v in [lmin, lmax], skipping the others.  A retry
// pass (c.wait = 0) defers a trade again whose dependency has not published,
// into the next pass's list.  The in-order pass (c.wait = 1, one list sorted
// by trade index, launched only when *ok, all sizes) waits instead: a
// dependency s < t is complete or deferred, and then it sits earlier in the
// list, claimed before t by a running CTA, so by induction every wait ends.
// Trades of at most 32 kWarpJ entries run on the CTA's first warp, up to
// 4 NT on the register path of the whole CTA, larger ones on the
// shared-memory path (a global slice above gen_max entries).
template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) k_phase_a_list(StepCtx c, const int32_t* __restrict__ list,
                                                                     int from_back, const unsigned long long* count,
                                                                     const int64_t* ok, unsigned long long* claim,
                                                                     int lmin, int lmax, int gen_max, char* gws,
                                                                     size_t slice) {
  using Ws = typename TeamCfg<NT>::Ws;
  extern __shared__ __align__(16) char sbuf[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ SelOut sel;
  __shared__ int64_t pick;
  if (ok && *reinterpret_cast<const volatile int64_t*>(ok) == 0) return;
  const int64_t nl = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(count));
  BlockTeam<NT> tm(red);
  for (;;) {
    if (threadIdx.x == 0) pick = static_cast<int64_t>(atomicAdd(claim, 1ull));
    __syncthreads();
    const int64_t p = pick;
    __syncthreads();
    if (p >= nl) return;
    const int64_t t = __ldcg(list + (from_back ? -1 - p : p));
    const TradeRows tr = trade_rows(c, t);
    const int L = tr.du + tr.dv;
    if (L < lmin || L > lmax) continue;
    if (L <= WarpWs::kLmax) {
      if (threadIdx.x < 32) {
        WarpTeam wt;
        phase_a_reg<WarpTeam, kWarpJ, kWarpB, true>(wt, c, t, WarpWs{sbuf});
      }
    } else if (L <= Ws::kLmax) {
      phase_a_reg<BlockTeam<NT>, kTeamJ, TeamCfg<NT>::B, false>(tm, c, t, Ws{sbuf});
    } else {
      char* wsb = sbuf;
      if (L > gen_max) {
        wsb = gws + slice * blockIdx.x;
        if (threadIdx.x == 0) atomicAdd(c.gws_count, 1ull);
      }
      phase_a(tm, c, t, carve_a(wsb, L), &sel);
    }
    __syncthreads();
  }
}

// A retry pass's small trades (list[0 .. *count)): every warp claims one at
// a time.
__global__ void __launch_bounds__(32 * kWarpWarps, 4) k_phase_a_list_warp(StepCtx c, const int32_t* __restrict__ list,
                                                                       const unsigned long long* count,
                                                                       unsigned long long* claim) {
  extern __shared__ __align__(16) char wsm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpWs w{wsm + WarpWs::kBytes * wid};
  WarpTeam tm;
  const int64_t nl = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(count));
  for (;;) {
    int64_t p = 0;
    if (lane == 0) p = static_cast<int64_t>(atomicAdd(claim, 1ull));
    p = static_cast<int64_t>(tm.bcast(static_cast<uint64_t>(p), 0));
    if (p >= nl) return;
    phase_a_reg<WarpTeam, kWarpJ, kWarpB, true>(tm, c, __ldcg(list + p), w);
  }
}

// The last pass's list of deferred trades (nsmall from the front, nbig
// from the back of list[0 .. cap)) gathered and sorted by index in one CTA
// into list[0 .. n), when n <= kSortListMax (*ok = 1, *n_out = n);
// otherwise *ok = 0 and the in-order pass scans the done flags instead.
constexpr int kSortListMax = 16384;   // 64 KB of dynamic shared memory
__global__ void __launch_bounds__(1024) k_sort_list(int32_t* list, int64_t cap, const unsigned long long* nsmall,
                                                    const unsigned long long* nbig, int64_t* ok, int64_t* n_out) {
  extern __shared__ __align__(16) int32_t a[];
  __shared__ int64_t red[BlockTeam<1024>::kRedSlots];
  const int64_t ns = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(nsmall));
  const int64_t nb = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(nbig));
  const int64_t nl = ns + nb;
  if (nl > kSortListMax) {
    if (threadIdx.x == 0) *ok = 0;
    return;
  }
  const int P = nl > 1 ? next_pow2(static_cast<int>(nl)) : 1;
  for (int i = threadIdx.x; i < P; i += 1024)
    a[i] = i < ns ? list[i] : i < nl ? list[cap - 1 - (i - ns)] : 0x7fffffff;
  __syncthreads();
  BlockTeam<1024> tm(red);
  team_bitonic_sort(tm, a, P);
  for (int i = threadIdx.x; i < nl; i += 1024) list[i] = a[i];
  if (threadIdx.x == 0) {
    *ok = 1;
    *n_out = nl;
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

namespace {
// Attributes of the kernels built in a one-graph and a general version.
template <bool kOneSeed>
int init_seed_kernels(Graph* h) {
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kMedThreads, kOneSeed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(block_smem_bytes(kBlockMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kBigThreads, kOneSeed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(block_smem_bytes(kSmemMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_team<kBigThreads, 512, kOneSeed>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(team_smem<kBigThreads, 512>())));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_team<kBigThreads, kBigThreads, kOneSeed>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(team_smem<kBigThreads, kBigThreads>())));
  // shared memory, not L1, limits how many CTAs of this kernel an SM holds
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_block<kMedThreads, kOneSeed>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
  return CB_OK;
}
}  // namespace

int init_trade_kernels(Graph* h) {
  // the largest dynamic shared memory any handle may ask of each kernel
  int rc = init_seed_kernels<true>(h);
  if (rc || (rc = init_seed_kernels<false>(h))) return rc;
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_inorder<kMedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(ws_a_bytes(kBlockMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_inorder<kBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(ws_a_bytes(kSmemMaxCap))));
  CB_CUDA(h, cudaFuncSetAttribute(k_sort_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kSortListMax * sizeof(int32_t))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_list<kMedThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(std::max(TeamCfg<kMedThreads>::Ws::kBytes,
                                                            ws_a_bytes(kBlockMaxCap)))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_list<kBigThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(std::max(TeamCfg<kBigThreads>::Ws::kBytes,
                                                            ws_a_bytes(kSmemMaxCap)))));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_lanes<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(LaneCfg<8>::kSmem)));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_lanes<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(LaneCfg<16>::kSmem)));
  // shared memory, not L1, limits how many CTAs of these kernels an SM holds
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_lanes<8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  CB_CUDA(h, cudaFuncSetAttribute(k_phase_a_lanes<16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  return CB_OK;
}

size_t trade_ws_slice_bytes(int64_t max_trade) {
  return (ws_a_bytes(static_cast<int>(max_trade)) + 255) & ~size_t(255);
}
size_t trade_smem_bytes(int entries) { return ws_a_bytes(entries); }

// Passes of the fix-up: enough that one pass's far-trade records (8 or 16
// bytes per trade) stay below kFixSliceBytes, or the "fix_passes" option.
constexpr int64_t kFixSliceBytes = int64_t(72) << 20;
int fix_passes(const Graph* h) {
  if (h->fix_passes > 0) return h->fix_passes;
  const int64_t rec = (h->n <= kNarrowPackMax && !h->wide_pack) ? 8 : 16;
  return static_cast<int>(std::max<int64_t>(1, (h->ntasks * rec + kFixSliceBytes - 1) / kFixSliceBytes));
}

int super_step(Graph* h) {
  if (h->g >= 0xfffffffeull) return fail(h, CB_ERANGE, "super-step counter exhausted");
  cudaStream_t s = h->stream;
  const int nxt = 1 - h->cur;
  const int eset = h->ev_set;
  cudaEvent_t* ev = h->ev[eset];
  if (h->timing && h->ev_pending[eset]) {
    const int frc = flush_timing(h, eset, true);
    if (frc) return frc;
  }
  if (h->timing) CB_CUDA(h, cudaEventRecord(ev[0], s));
  int rc = prepare_next(h);
  if (rc) return rc;
  if (h->timing) CB_CUDA(h, cudaEventRecord(ev[1], s));
  StepCtx c;
  c.n = h->n;
  c.T = h->T;
  c.stamp = 1;   // done flags are cleared at the start of every step
  c.segs = h->segs;
  c.seg_of = h->seg_of;
  c.rp = h->rp[h->cur];
  c.col = h->col[h->cur];
  c.fb = h->stash;
  c.ph = h->col[nxt];
  c.Minv = h->Minv;
  c.thr_key = h->thr_key;
  c.thr_tb = h->thr_tb;
  c.thr_top = h->thr_top;
  c.done = h->done;
  c.err = h->err;
  c.M = h->M;
  c.rp_next = h->rp[nxt];
  philox_round_keys(h->hsegs[0].seed, c.ks);   // used only when the handle holds one graph
  // counters (kCtr* in cb_internal.cuh): class lists, the first pass's class
  // sizes, deferrals per pass, chunks claimed by the in-order pass,
  // global-workspace trades
  int64_t* cnt = h->counters;
  unsigned long long* ucnt = reinterpret_cast<unsigned long long*>(cnt);
  c.gws_count = ucnt + kCtrGws;
  CB_CUDA(h, cudaMemsetAsync(cnt, 0, kCounters * sizeof(int64_t), s));
  const int64_t ntasks = h->ntasks;
  if (ntasks == 0) return finish_step(h);
  CB_CUDA(h, cudaMemsetAsync(h->done, 0, sizeof(uint32_t) * ntasks, s));
  const int tile_max = h->tile_paths ? std::min(h->tile_max, kTileMaxCap) : 0;
  const int block_max = std::max(h->block_max, tile_max);
  // size classes: warp (L <= tile_max), teams of 64 / 128 / 256 threads (up
  // to 256 / 512 / block_max <= 1024 entries), of 512 / 1024 threads in a
  // 1024-thread CTA (up to 2048 / min(4096, smem_max)), and the largest
  // trades on the shared-memory kernel; "cta_paths" 0 sends everything above
  // the warp class to the shared-memory kernels (256 threads up to
  // block_max, 1024 above)
  ClassTh th;
  {
    const int lreg = std::min(TeamCfg<kBigThreads>::kMax, h->smem_max);
    const int t3 = h->cta_paths ? std::max(tile_max, std::min(block_max, TeamCfg<256>::kMax)) : block_max;
    const int t5 = h->cta_paths ? std::max(t3, lreg) : t3;
    // lane teams of 8 / 16 (L <= 32 / 64), a warp (L <= tile_max), teams of
    // 64 .. 1024 threads, the 1024-thread shared-memory kernel
    th.th[0] = h->lane_teams ? std::min(LaneCfg<8>::Ws::kLmax, tile_max) : 0;
    th.th[1] = h->lane_teams ? std::min(LaneCfg<16>::Ws::kLmax, tile_max) : 0;
    th.th[2] = tile_max;
    th.th[3] = h->cta_paths ? std::min(std::max(TeamCfg<64>::kMax, tile_max), t3) : tile_max;
    th.th[4] = h->cta_paths ? std::min(std::max(TeamCfg<128>::kMax, th.th[3]), t3) : tile_max;
    th.th[5] = t3;
    th.th[6] = h->cta_paths ? std::min(std::max(TeamCfg<512>::kMax, t3), t5) : t3;
    th.th[7] = t5;
  }
  auto grid_n = [&](int64_t work) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, h->num_sms * 8)));
  };
  const size_t med_smem = ws_a_bytes(std::max(block_max, 1));      // in-order pass (no staging)
  const size_t big_smem = ws_a_bytes(std::max(h->smem_max, 1));
  const size_t med_smem_st = block_smem_bytes(std::max(block_max, 1));   // threshold kernels with staging
  const size_t big_smem_st = block_smem_bytes(std::max(h->smem_max, 1));
  const unsigned mgrid = static_cast<unsigned>(h->num_sms * 4);
  const unsigned bgrid = static_cast<unsigned>(std::max(1, std::min(h->num_sms, h->ws_ctas)));
  const unsigned sgrid = static_cast<unsigned>(h->num_sms);
  char* gws = static_cast<char*>(h->ws_global);
  c.wait = 0;
  c.cand_max = h->cand_max;
  c.wait_ns = h->wait_ns;
  c.hold_publish = h->hold_publish;
  const int32_t* L = h->lists;
  auto launched = [&]() -> int {
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    return CB_OK;
  };
  // class lists (every trade, or only the deferred ones): a stable counting
  // sort of the trades by class
  auto classify = [&](int only_deferred) -> int {
    const int64_t nch = (ntasks + kClassChunk - 1) / kClassChunk;
    const unsigned cgrid = static_cast<unsigned>(std::min<int64_t>(nch, int64_t(h->num_sms) * 8));
    k_class_count<<<cgrid, kClassThreads, 0, s>>>(c, ntasks, th, nch, only_deferred, h->cls_flag, cnt);
    int r = launched();
    if (r) return r;
    CB_CUDA(h, exclusive_scan_i32(h->cls_flag, h->cls_scan, kClasses * nch, h->scan_ws, s, &h->launches));
    k_class_place<<<cgrid, kClassThreads, 0, s>>>(c, ntasks, th, nch, only_deferred, h->cls_scan, h->lists);
    if ((r = launched())) return r;
    k_class_bounds<<<1, 32, 0, s>>>(h->cls_scan, nch, !only_deferred, cnt);
    return launched();
  };
  // one pass of every class's kernel; a trade whose dependency has not
  // published yet is (again) marked deferred
  // with "timing" on, the first pass brackets each class's kernel with
  // events ev[4 + k] .. ev[5 + k] (a class without its own kernel takes none)
  bool time_classes = false;
  auto mark = [&](int k) -> int {
    if (time_classes) CB_CUDA(h, cudaEventRecord(ev[4 + k], s));
    return CB_OK;
  };
  const unsigned wgrid = static_cast<unsigned>(h->num_sms * 8);
  // the team and shared-memory kernels come in a one-graph version (the
  // seed's Philox round keys in the kernel parameters) and a general one
  auto run_classes_as = [&](auto one_seed) -> int {
    constexpr bool kOne = decltype(one_seed)::value;
    int r;
    if ((r = mark(0))) return r;
    if (h->lane_teams) {
      k_phase_a_lanes<8><<<wgrid, 32 * kWarpWarps, LaneCfg<8>::kSmem, s>>>(c, L, cnt, 0);
      if ((r = launched()) || (r = mark(1))) return r;
      k_phase_a_lanes<16><<<wgrid, 32 * kWarpWarps, LaneCfg<16>::kSmem, s>>>(c, L, cnt, 1);
      if ((r = launched()) || (r = mark(2))) return r;
    } else if ((r = mark(1)) || (r = mark(2))) {
      return r;
    }
    k_phase_a_warp<<<wgrid, 32 * kWarpWarps, WarpWs::kBytes * kWarpWarps, s>>>(c, L, cnt, 2);
    if ((r = launched()) || (r = mark(3))) return r;
    if (h->cta_paths) {
      k_phase_a_team<256, 64, kOne><<<mgrid, 256, team_smem<256, 64>(), s>>>(c, L, cnt, 3);
      if ((r = launched()) || (r = mark(4))) return r;
      k_phase_a_team<256, 128, kOne><<<mgrid, 256, team_smem<256, 128>(), s>>>(c, L, cnt, 4);
      if ((r = launched()) || (r = mark(5))) return r;
      k_phase_a_team<256, 256, kOne><<<mgrid, 256, team_smem<256, 256>(), s>>>(c, L, cnt, 5);
      if ((r = launched()) || (r = mark(6))) return r;
      k_phase_a_team<kBigThreads, 512, kOne><<<sgrid, kBigThreads, team_smem<kBigThreads, 512>(), s>>>(c, L, cnt,
                                                                                                      6);
      if ((r = launched()) || (r = mark(7))) return r;
      k_phase_a_team<kBigThreads, kBigThreads, kOne>
          <<<sgrid, kBigThreads, team_smem<kBigThreads, kBigThreads>(), s>>>(c, L, cnt, 7);
      if ((r = launched()) || (r = mark(8))) return r;
    } else {
      k_phase_a_block<kMedThreads, kOne><<<mgrid, kMedThreads, med_smem_st, s>>>(c, L, cnt, 5, block_max, gws,
                                                                                h->ws_slice, block_max);
      if ((r = launched())) return r;
      for (int k = 4; k <= 8; ++k)
        if ((r = mark(k))) return r;
    }
    // the largest trades: 1024 threads, up to smem_max entries in shared
    // memory (staged by a bulk copy), a global-memory slice above
    k_phase_a_block<kBigThreads, kOne><<<bgrid, kBigThreads, big_smem_st, s>>>(c, L, cnt, 8, h->smem_max, gws,
                                                                              h->ws_slice, h->smem_max);
    if ((r = launched())) return r;
    return mark(9);
  };
  auto run_classes = [&]() -> int {
    return c.seg_of ? run_classes_as(std::false_type{}) : run_classes_as(std::true_type{});
  };
  // the first pass over every trade, then retry_passes parallel passes over
  // the deferred ones: each runs every deferred trade whose dependencies
  // have published by then, so chains of dependent trades shrink by a level
  // per pass.  Pass r counts its deferrals in ctr[kCtrPassLeft + r] and lists
  // them in dlist[r & 1] for pass r + 1: the small ones from the front
  // (ctr[kCtrPassSmall + r] of them), the others from the back
  // (ctr[kCtrPassBig + r]).
  auto list_for = [&](int r) {
    c.def_count = ucnt + kCtrPassLeft + r;
    c.def_list = h->dlist + (r & 1) * ntasks;
    c.def_small = ucnt + kCtrPassSmall + r;
    c.def_big = ucnt + kCtrPassBig + r;
    c.def_cap = ntasks;
  };
  time_classes = h->timing;
  list_for(0);
  if ((rc = classify(0)) || (rc = run_classes())) return rc;
  time_classes = false;
  const unsigned lgrid = static_cast<unsigned>(gws ? std::min(h->num_sms * 4, h->ws_ctas) : h->num_sms * 4);
  const size_t list_smem = std::max(TeamCfg<kMedThreads>::Ws::kBytes, ws_a_bytes(std::max(block_max, 1)));
  const size_t list_smem_big = std::max(TeamCfg<kBigThreads>::Ws::kBytes, ws_a_bytes(std::max(h->smem_max, 1)));
  for (int r = 0; r < h->retry_passes; ++r) {
    // small trades on warps, medium on 256-thread CTAs, the largest on
    // 1024-thread CTAs (shared memory up to smem_max entries)
    const int32_t* in = h->dlist + (r & 1) * ntasks;
    list_for(r + 1);
    k_phase_a_list_warp<<<wgrid, 32 * kWarpWarps, WarpWs::kBytes * kWarpWarps, s>>>(c, in, ucnt + kCtrPassSmall + r,
                                                                                  ucnt + kCtrListClaim + 3 * r);
    CB_CUDA(h, cudaGetLastError());
    k_phase_a_list<kMedThreads><<<lgrid, kMedThreads, list_smem, s>>>(
        c, in + ntasks, 1, ucnt + kCtrPassBig + r, nullptr, ucnt + kCtrListClaim + 3 * r + 1, kListSmall + 1,
        TeamCfg<kMedThreads>::kMax, block_max, gws, h->ws_slice);
    CB_CUDA(h, cudaGetLastError());
    k_phase_a_list<kBigThreads><<<bgrid, kBigThreads, list_smem_big, s>>>(
        c, in + ntasks, 1, ucnt + kCtrPassBig + r, nullptr, ucnt + kCtrListClaim + 3 * r + 2,
        TeamCfg<kMedThreads>::kMax + 1, 0x7fffffff, h->smem_max, gws, h->ws_slice);
    CB_CUDA(h, cudaGetLastError());
    h->launches += 3;
  }
  if (h->timing) CB_CUDA(h, cudaEventRecord(ev[5 + kClasses], s));
  // last pass: the trades still deferred, in index order, waiting on
  // dependencies: over the last list sorted by index when it holds at most
  // kSortListMax trades, else by scanning every trade's done flag.
  // 1024-thread CTAs keep large trades in shared memory; 256-thread CTAs
  // (four per SM) run many small deferred trades at once, large ones from a
  // global slice.
  {
    const int R = h->retry_passes;
    int32_t* last = h->dlist + (R & 1) * ntasks;
    int64_t* ok = cnt + kCtrListOk;
    const unsigned long long* nlast = ucnt + kCtrListN;
    k_sort_list<<<1, 1024, kSortListMax * sizeof(int32_t), s>>>(last, ntasks, ucnt + kCtrPassSmall + R,
                                                               ucnt + kCtrPassBig + R, ok, cnt + kCtrListN);
    CB_CUDA(h, cudaGetLastError());
    ++h->launches;
    c.wait = 1;
    c.def_count = ucnt + kCtrPassLeft + R + 1;   // a wait that ran out leaves its trade deferred
    c.def_list = nullptr;
    unsigned long long* lclaim = ucnt + kCtrListClaim + 3 * kRetryPassesMax;
    if (h->inorder_threads == kBigThreads) {
      k_phase_a_list<kBigThreads><<<bgrid, kBigThreads, list_smem_big, s>>>(c, last, 0, nlast, ok, lclaim, 0,
                                                                           0x7fffffff, h->smem_max, gws, h->ws_slice);
      CB_CUDA(h, cudaGetLastError());
      const int64_t chunk = std::max<int64_t>(1024, (ntasks + int64_t(bgrid) * 8 - 1) / (int64_t(bgrid) * 8));
      k_phase_a_inorder<kBigThreads><<<bgrid, kBigThreads, big_smem, s>>>(c, ntasks, chunk, ucnt + kCtrClaims,
                                                                         h->smem_max, gws, h->ws_slice, ok);
      CB_CUDA(h, cudaGetLastError());
    } else {
      k_phase_a_list<kMedThreads><<<lgrid, kMedThreads, list_smem, s>>>(c, last, 0, nlast, ok, lclaim, 0, 0x7fffffff,
                                                                       block_max, gws, h->ws_slice);
      CB_CUDA(h, cudaGetLastError());
      const int64_t chunk = std::max<int64_t>(512, (ntasks + int64_t(lgrid) * 4 - 1) / (int64_t(lgrid) * 4));
      k_phase_a_inorder<kMedThreads><<<lgrid, kMedThreads, med_smem, s>>>(c, ntasks, chunk, ucnt + kCtrClaims,
                                                                         block_max, gws, h->ws_slice, ok);
      CB_CUDA(h, cudaGetLastError());
    }
    h->launches += 2;
  }
  if (h->timing) CB_CUDA(h, cudaEventRecord(ev[2], s));
  // rebuild: far-trade records, each chunk's first row, then the fix-up in
  // passes over slices of the far trades; its output overwrites this step's
  // adjacency, which phase A no longer needs, and becomes step g+1's
  {
    const int64_t nnz = h->nnz;
    const int64_t nchunks = (nnz + kFixChunk - 1) / kFixChunk;
    int32_t* chunk_row = h->cls_flag;   // nchunks + 1 entries, free after the classification
    if (nchunks > 0) {
      const bool narrow = h->n <= kNarrowPackMax && !h->wide_pack;
      if (narrow) k_far_pack<true><<<grid_n(ntasks), 256, 0, s>>>(c, ntasks, h->far_pack);
      else k_far_pack<false><<<grid_n(ntasks), 256, 0, s>>>(c, ntasks, h->far_pack);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
      k_chunk_rows<<<grid_n(h->n), 256, 0, s>>>(h->n, c.rp_next, nchunks, chunk_row);
      CB_CUDA(h, cudaGetLastError());
      ++h->launches;
      const int passes = fix_passes(h);
      const int64_t per = (ntasks + passes - 1) / passes;
      const unsigned fgrid = static_cast<unsigned>(std::min<int64_t>(nchunks, int64_t(h->num_sms) * 4));
      int32_t* out = h->col[h->cur];
      for (int q = 0; q < passes; ++q) {
        const uint32_t lo = static_cast<uint32_t>(std::min<int64_t>(ntasks, q * per));
        const uint32_t hi = static_cast<uint32_t>(std::min<int64_t>(ntasks, (q + 1) * per));
        const bool last = q == passes - 1;
        auto fk = narrow ? (last ? k_fixup<true, true> : k_fixup<true, false>)
                         : (last ? k_fixup<false, true> : k_fixup<false, false>);
        fk<<<fgrid, kFixThreads, 0, s>>>(c, nnz, lo, hi, c.ph, c.fb, out, h->far_pack, chunk_row);
        CB_CUDA(h, cudaGetLastError());
        ++h->launches;
      }
    }
    std::swap(h->col[0], h->col[1]);   // the step's output is now the other side of the ping-pong
  }
  if (h->timing) {
    CB_CUDA(h, cudaEventRecord(ev[3], s));
    h->ev_pending[eset] = true;
    h->ev_set = 1 - eset;
  }
  return finish_step(h);
}

int flush_timing(Graph* h, int set, bool add) {
  if (!h->ev_pending[set]) return CB_OK;
  h->ev_pending[set] = false;
  cudaEvent_t* ev = h->ev[set];
  CB_CUDA(h, cudaEventSynchronize(ev[3]));
  if (!add) return CB_OK;
  float a = 0, b = 0, d = 0, tot = 0;
  CB_CUDA(h, cudaEventElapsedTime(&a, ev[0], ev[1]));
  CB_CUDA(h, cudaEventElapsedTime(&b, ev[1], ev[2]));
  CB_CUDA(h, cudaEventElapsedTime(&d, ev[2], ev[3]));
  CB_CUDA(h, cudaEventElapsedTime(&tot, ev[0], ev[3]));
  h->phase_ms[0] += a;
  h->phase_ms[1] += b;
  h->phase_ms[2] += d;
  h->phase_ms[3] += tot;
  for (int k = 0; k < kClasses; ++k) {
    float e = 0;
    CB_CUDA(h, cudaEventElapsedTime(&e, ev[4 + k], ev[5 + k]));
    h->phase_ms[4 + k] += e;
  }
  float re = 0, io = 0;
  CB_CUDA(h, cudaEventElapsedTime(&re, ev[4 + kClasses], ev[5 + kClasses]));
  CB_CUDA(h, cudaEventElapsedTime(&io, ev[5 + kClasses], ev[2]));
  h->phase_ms[4 + kClasses] += re;
  h->phase_ms[5 + kClasses] += io;
  return CB_OK;
}

}  // namespace cb
