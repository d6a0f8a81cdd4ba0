// Uniform single trades (Simple Undirected Curveball, Section 3.2) on the
// device, and the successor lists Suc of a trade sequence (Section 4.1).
//
// The sequence runs as a dataflow in the manner of EM-CB / IM-CB (Sections
// 4.1-4.2), in the position space of the handle's current super step:
//   - Suc gives, for every (trade, endpoint), the endpoint's next trade, and
//     for every node its first trade.
//   - Every edge waits in an inbox of the next trade of either endpoint:
//     that trade is the only one that can change it.
//   - An inbox entry carries the neighbour and the neighbour's next trade.
//     Trade k's inbox for node x has deg(x) slots, reserved by one 64-bit
//     atomic per entry (both sides' counts packed).
//   - The reservation that fills the last slot queues the trade.
//   - Persistent CTAs take queued trades in queue order. Each one:
//       - gathers both inboxes, waiting (bounded) for entries still being
//         written;
//       - finds the common and disjoint neighbours through a hash of u's
//         neighbours;
//       - finds the threshold of sigma(D) by a radix select on D's keys;
//       - sends every resulting edge on.
//   - An edge whose endpoints both have no further trade goes to its rows of
//     the output.
// The critical path of the dataflow is a chain of dependent trades. So a
// trade's own latency counts: no sort, few barriers, and the atomics of a
// thread's messages in flight together.
// Every trade sees exactly the neighbourhoods it would see in index order:
// an edge {a, b} changes only in trades of a or b, and it reaches the first
// of those before anything else touches it.
#include <algorithm>
#include <cstring>

#include "cb_internal.cuh"
#include "philox.cuh"
#include "team.cuh"

namespace cb {

struct UniBufs {
  int64_t cap_trades = 0;      // trades per chunk the buffers hold
  int64_t n = 0;
  int32_t* tp = nullptr;       // 2L: positions of u_i (even) and v_i (odd)
  int32_t* dslot = nullptr;    // 2L: degree of each slot's node (scan input)
  int64_t* ib = nullptr;       // 2L+1: first inbox entry of each slot
  int32_t* suc = nullptr;      // 2L: slot ids grouped by node, increasing
  int32_t* nxt = nullptr;      // 2L: next trade of the slot's node after its trade
  unsigned long long* fill = nullptr;   // L: inbox counts (side 0 low, side 1 high)
  int32_t* queue = nullptr;    // L: runnable trades; small ones from the front, big ones from the back
  int32_t* occ = nullptr;      // n: occurrences, then fill cursors
  int64_t* sbeg = nullptr;     // n+1: Suc offsets
  int32_t* ocur = nullptr;     // n: output row cursors
  unsigned long long* ctr = nullptr;   // run queue head and tail, a cache line apart
  void* scan_ws = nullptr;
  int2* inbox = nullptr;
  int64_t inbox_cap = 0;
  char* gslice = nullptr;      // per-CTA work space for trades above the shared-memory cap
  int64_t slice_elems = 0;
  int ctas = 0;
  size_t bytes = 0, inbox_bytes = 0, slice_bytes = 0;
};

namespace {

constexpr int32_t kInf = 0x7fffffff;            // no further trade
// Executor CTAs of NT = 256 (two per SM), 512 or 1024 threads (option
// "uniform_threads"): larger CTAs give a hub trade more threads but keep
// fewer trades running at once.
template <int NT>
constexpr int uni_smem_elems() { return NT == 1024 ? 4096 : 2048; }   // trades up to this many entries in shared memory
constexpr int64_t kUniChunkMin = 65536;

__device__ __forceinline__ void latch(int32_t* err, int32_t code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

__device__ __forceinline__ int2 ld_relaxed_v2(const int2* p) {
  int2 v;
  asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_v2(int2* p, int32_t x, int32_t y) {
  asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(x), "r"(y) : "memory");
}

__device__ __forceinline__ void st_relaxed_i32(int32_t* p, int32_t x) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

__device__ __forceinline__ int32_t ld_relaxed_i32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------- the sequence

// Pair of trade i on n >= 2 nodes: counter (i_lo, i_hi, 0, 5), multiply-high
// maps of words 0 and 1 (see cb_uniform.h).
__device__ __forceinline__ void uniform_pair(uint64_t seed, int64_t n, uint64_t i, int32_t* u, int32_t* v) {
  const Philox4 r = philox4x32_10(static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), 0u, 5u, seed);
  const int64_t a = static_cast<int64_t>((static_cast<uint64_t>(r.w0) * static_cast<uint64_t>(n)) >> 32);
  const int64_t w = static_cast<int64_t>((static_cast<uint64_t>(r.w1) * static_cast<uint64_t>(n - 1)) >> 32);
  *u = static_cast<int32_t>(a);
  *v = static_cast<int32_t>(w + (w >= a));
}

// pairs of trades first..first+count-1; mapped through pos (node id ->
// position) when given; with rp, each slot's degree goes to dslot.
__global__ void k_uni_draw(int64_t count, uint64_t first, uint64_t seed, int64_t n, const int32_t* __restrict__ pos,
                           const int64_t* __restrict__ rp, int32_t* __restrict__ out, int32_t* __restrict__ dslot) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    int32_t u, v;
    uniform_pair(seed, n, first + static_cast<uint64_t>(i), &u, &v);
    if (pos) {
      u = pos[u];
      v = pos[v];
    }
    out[2 * i] = u;
    out[2 * i + 1] = v;
    if (dslot) {
      dslot[2 * i] = static_cast<int32_t>(rp[u + 1] - rp[u]);
      dslot[2 * i + 1] = static_cast<int32_t>(rp[v + 1] - rp[v]);
    }
  }
}

// occ[x] = number of slots naming x; pairs out of range or with equal nodes latch err.
__global__ void k_uni_count(int64_t count, int64_t n, const int32_t* __restrict__ tp, int32_t* __restrict__ occ,
                            int32_t* err) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = tp[2 * i], b = tp[2 * i + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) {
      latch(err, kErrValidate);
      continue;
    }
    atomicAdd(&occ[a], 1);
    atomicAdd(&occ[b], 1);
  }
}

// suc[sbeg[x] + k] = slot ids of x (unordered; cursors start at 0)
__global__ void k_uni_fill(int64_t slots, const int32_t* __restrict__ tp, const int64_t* __restrict__ sbeg,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ suc) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < slots; j += int64_t(gridDim.x) * blockDim.x) {
    const int32_t x = tp[j];
    const int32_t k = atomicAdd(&cursor[x], 1);
    suc[sbeg[x] + k] = static_cast<int32_t>(j);
  }
}

// Each node's slot list in increasing order (a node is in a trade at most
// once, so slot order is trade order); with nxt, every slot's next trade.
__global__ void k_uni_sort(int64_t n, const int64_t* __restrict__ sbeg, int32_t* __restrict__ suc,
                           int32_t* __restrict__ nxt) {
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = sbeg[x], e = sbeg[x + 1];
    for (int64_t i = b + 1; i < e; ++i) {   // lists are short: Poisson(2L/n) long
      const int32_t key = suc[i];
      int64_t j = i - 1;
      while (j >= b && suc[j] > key) {
        suc[j + 1] = suc[j];
        --j;
      }
      suc[j + 1] = key;
    }
    if (nxt)
      for (int64_t i = b; i < e; ++i) nxt[suc[i]] = (i + 1 < e) ? (suc[i + 1] >> 1) : kInf;
  }
}

__global__ void k_uni_trade_index(int64_t slots, const int32_t* __restrict__ suc, int32_t* __restrict__ out) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < slots; j += int64_t(gridDim.x) * blockDim.x)
    out[j] = suc[j] >> 1;
}

// ------------------------------------------------------------- the dataflow

struct UniCtx {
  int64_t L;                 // trades in this chunk
  uint64_t first;            // global index of the chunk's first trade
  uint64_t seed;
  const int64_t* rp;         // position-space row offsets (degrees never change)
  const int32_t* order;      // node id at each position (keys use ids)
  const int32_t* tp;
  const int32_t* nxt;
  const int64_t* ib;
  const int64_t* sbeg;
  const int32_t* suc;
  int2* inbox;
  unsigned long long* fill;
  int32_t* queue;
  unsigned long long* ctr;
  int32_t* ocur;
  int32_t* col_out;
  int32_t* err;
  char* gslice;
  int64_t slice_elems;
  unsigned long long* swaps;   // (performed, possible) swap counts, or null
  uint64_t wait_ns;            // longest single wait (run queue, inbox entry)
  int64_t hold_trade;          // test hook: messages to this trade of the chunk are dropped (-1: none)
};

// The run queue: a ticket (kHead) takes the next slot, a push (kTail)
// fills the next slot; the two counters sit on different cache lines.
// Every trade is queued exactly once, so every ticket below L ends.
constexpr int kHead = 0, kTail = 16, kCtrWords = 32;

__device__ __forceinline__ void push(const UniCtx& c, int64_t k) {
  const unsigned long long q = atomicAdd(&c.ctr[kTail], 1ull);
  if (q >= static_cast<unsigned long long>(c.L)) {
    latch(c.err, kErrUniform);
    return;
  }
  st_relaxed_i32(c.queue + q, static_cast<int32_t>(k));
}

// The next queued trade, or -1 when every slot is taken or a wait gave up.
__device__ int64_t take_ticket(const UniCtx& c) {
  const unsigned long long q = atomicAdd(&c.ctr[kHead], 1ull);
  if (q >= static_cast<unsigned long long>(c.L)) return -1;
  int32_t t = ld_relaxed_i32(c.queue + q);
  if (t < 0) {
    const uint64_t t0 = globaltimer();
    for (;;) {
      __nanosleep(200);
      t = ld_relaxed_i32(c.queue + q);
      if (t >= 0) break;
      if (ld_volatile_i32(c.err) != 0) return -1;
      if (globaltimer() - t0 > c.wait_ns) {
        latch(c.err, kErrUniformWait);
        return -1;
      }
    }
  }
  return t;
}

// Append (other, other_tau) to node x's inbox at trade d.
__device__ void append(const UniCtx& c, int32_t d, int32_t x, int32_t other, int32_t other_tau) {
  if (d == c.hold_trade) return;   // test hook: the trade never becomes runnable
  const int32_t a = c.tp[2 * int64_t(d)], b = c.tp[2 * int64_t(d) + 1];
  const int side = (x == a) ? 0 : 1;
  if (x != a && x != b) {
    latch(c.err, kErrUniform);
    return;
  }
  const uint64_t du = static_cast<uint64_t>(c.rp[a + 1] - c.rp[a]), dv = static_cast<uint64_t>(c.rp[b + 1] - c.rp[b]);
  const unsigned long long inc = side ? (1ull << 32) : 1ull;
  const unsigned long long old = atomicAdd(&c.fill[d], inc);
  const uint64_t slot = side ? (old >> 32) : (old & 0xffffffffull);
  if (slot >= (side ? dv : du)) {
    latch(c.err, kErrUniform);
    return;
  }
  st_relaxed_v2(c.inbox + c.ib[2 * int64_t(d) + side] + slot, other, other_tau);
  if (old + inc == ((dv << 32) | du)) push(c, d);
}

// The edge {a, b} into its rows of the output.
__device__ void commit(const UniCtx& c, int32_t a, int32_t b) {
  const int64_t ba = c.rp[a], bb = c.rp[b];
  const int32_t sa = atomicAdd(&c.ocur[a], 1), sb = atomicAdd(&c.ocur[b], 1);
  if (sa < c.rp[a + 1] - ba) c.col_out[ba + sa] = b;
  else latch(c.err, kErrRowLength);
  if (sb < c.rp[b + 1] - bb) c.col_out[bb + sb] = a;
  else latch(c.err, kErrRowLength);
}

// The edge {a, b}, a's next trade ta, b's next trade tb: to the earlier of
// the two (both inboxes when they are the same trade), or out.
__device__ void route(const UniCtx& c, int32_t a, int32_t ta, int32_t b, int32_t tb) {
  const int32_t d = min(ta, tb);
  if (d == kInf) {
    commit(c, a, b);
    return;
  }
  if (ta == d) append(c, d, a, b, tb);
  if (tb == d) append(c, d, b, a, ta);
}

__device__ __forceinline__ int32_t first_trade(const UniCtx& c, int32_t x) {
  const int64_t b = c.sbeg[x];
  return b < c.sbeg[x + 1] ? (c.suc[b] >> 1) : kInf;
}

// Every edge of the input to the first trade of either endpoint; trades with
// no entries to wait for are queued here.
__global__ void k_uni_route(UniCtx c, int64_t n, const int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t a = gw; a < n; a += nw) {
    const int64_t b0 = c.rp[a], b1 = c.rp[a + 1];
    if (b0 == b1) continue;
    const int32_t ta = first_trade(c, static_cast<int32_t>(a));
    for (int64_t q = b0 + lane; q < b1; q += 32) {
      const int32_t b = col[q];
      if (b > a) route(c, static_cast<int32_t>(a), ta, b, first_trade(c, b));
    }
  }
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < c.L; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = c.tp[2 * k], b = c.tp[2 * k + 1];
    if (c.rp[a + 1] == c.rp[a] && c.rp[b + 1] == c.rp[b]) push(c, k);
  }
}

// Bounded wait for an inbox entry still being written (the cold path).
__device__ __noinline__ bool wait_entry(const int2* p, const int32_t* err, uint64_t wait_ns, int2* out) {
  int2 m = ld_relaxed_v2(p);
  if (m.x != -1) {
    *out = m;
    return true;
  }
  const uint64_t t0 = globaltimer();
  for (;;) {
    __nanosleep(100);
    m = ld_relaxed_v2(p);
    if (m.x != -1) {
      *out = m;
      return true;
    }
    if (ld_volatile_i32(err) != 0 || globaltimer() - t0 > wait_ns) return false;
  }
}

// Per-trade work space: the gathered entries (neighbour, its next trade),
// their shuffle keys, flags and a hash of u's neighbours.
template <class HT>
struct TradeWs {
  int2* ent;
  uint64_t* key;
  HT* hash;        // entry index + 1 of u's neighbours, 0 = empty
  uint8_t* flag;   // bit 0 side (0: u's inbox, 1: v's), bit 1 common, bit 2 the edge {u, v}, bit 3 to u
};

// Big trades keep their entries in global memory but hash u's neighbours in
// the (then unused) shared memory with 16-bit slots, up to this degree of u
// at a load factor of at most 3/4.
constexpr int kHash16MaxDu = 12288;

constexpr size_t kWsBytesPerElem = sizeof(int2) + sizeof(uint64_t) + 2 * sizeof(int32_t) + 1;

__device__ __forceinline__ TradeWs<int32_t> carve_ws(char* base, int64_t cap) {
  TradeWs<int32_t> w;
  w.ent = reinterpret_cast<int2*>(base);
  w.key = reinterpret_cast<uint64_t*>(base + sizeof(int2) * cap);
  w.hash = reinterpret_cast<int32_t*>(base + (sizeof(int2) + sizeof(uint64_t)) * cap);
  w.flag = reinterpret_cast<uint8_t*>(base + (sizeof(int2) + sizeof(uint64_t) + 2 * sizeof(int32_t)) * cap);
  return w;
}

// log2 of the smallest power of two >= max(want, 2)
__device__ __forceinline__ int hash_bits(int64_t want) {
  int b = 1;
  while ((int64_t(1) << b) < want) ++b;
  return b;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t x, int hbits) {
  return (static_cast<uint32_t>(x) * 0x9E3779B1u) >> (32 - hbits);
}

// One message: the edge {a, b} with a's next trade ta and b's next trade tb.
// reserve() takes the slots (one atomic per message), deliver() writes them.
struct Msg {
  int32_t a, ta, b, tb, d;
  unsigned long long old;   // previous inbox counts of trade d, or the two row cursors
};

__device__ __forceinline__ void reserve(const UniCtx& c, Msg& m) {
  m.d = min(m.ta, m.tb);
  if (m.d == kInf) {
    const uint32_t sa = static_cast<uint32_t>(atomicAdd(&c.ocur[m.a], 1));
    const uint32_t sb = static_cast<uint32_t>(atomicAdd(&c.ocur[m.b], 1));
    m.old = (static_cast<unsigned long long>(sb) << 32) | sa;
    return;
  }
  const int32_t x0 = c.tp[2 * int64_t(m.d)];
  unsigned long long inc = 0;
  if (m.ta == m.d) inc += (m.a == x0) ? 1ull : (1ull << 32);
  if (m.tb == m.d) inc += (m.b == x0) ? 1ull : (1ull << 32);
  m.old = atomicAdd(&c.fill[m.d], inc);
}

__device__ void deliver_one(const UniCtx& c, int32_t d, int side, uint64_t slot, uint64_t cap, int32_t other,
                            int32_t other_tau) {
  if (slot >= cap) {
    latch(c.err, kErrUniform);
    return;
  }
  st_relaxed_v2(c.inbox + c.ib[2 * int64_t(d) + side] + slot, other, other_tau);
}

__device__ void deliver(const UniCtx& c, const Msg& m) {
  if (m.d == kInf) {
    const int64_t ba = c.rp[m.a], bb = c.rp[m.b];
    const uint32_t sa = static_cast<uint32_t>(m.old), sb = static_cast<uint32_t>(m.old >> 32);
    if (sa < c.rp[m.a + 1] - ba) c.col_out[ba + sa] = m.b;
    else latch(c.err, kErrRowLength);
    if (sb < c.rp[m.b + 1] - bb) c.col_out[bb + sb] = m.a;
    else latch(c.err, kErrRowLength);
    return;
  }
  const int64_t d = m.d;
  const int32_t x0 = c.tp[2 * d], x1 = c.tp[2 * d + 1];
  const uint64_t du = static_cast<uint64_t>(c.rp[x0 + 1] - c.rp[x0]), dv = static_cast<uint64_t>(c.rp[x1 + 1] - c.rp[x1]);
  unsigned long long inc = 0;
  const uint64_t s0 = m.old & 0xffffffffull, s1 = m.old >> 32;
  if (m.ta == m.d) {
    if (m.a != x0 && m.a != x1) latch(c.err, kErrUniform);
    const int side = m.a == x0 ? 0 : 1;
    deliver_one(c, m.d, side, side ? s1 : s0, side ? dv : du, m.b, m.tb);
    inc += side ? (1ull << 32) : 1ull;
  }
  if (m.tb == m.d) {
    if (m.b != x0 && m.b != x1) latch(c.err, kErrUniform);
    const int side = m.b == x0 ? 0 : 1;
    deliver_one(c, m.d, side, side ? s1 : s0, side ? dv : du, m.a, m.ta);
    inc += side ? (1ull << 32) : 1ull;
  }
  if (m.old + inc == ((dv << 32) | du)) push(c, d);
}

// Elements of D with the same full key as entry e and a smaller node id
// (ties of 64-bit keys: practically never, hence the plain loop).
__device__ __noinline__ int tied_before(const UniCtx& c, const int2* ent, const uint64_t* key, const uint8_t* flag,
                                        int E, int e) {
  const uint32_t id = static_cast<uint32_t>(c.order[ent[e].x]);
  int before = 0;
  for (int q = 0; q < E; ++q)
    if ((flag[q] & 6) == 0 && key[q] == key[e] && static_cast<uint32_t>(c.order[ent[q].x]) < id) ++before;
  return before;
}

// messages per thread with their atomics in flight together (one in the
// 1024-thread executor, whose threads have 64 registers)
template <int NT>
constexpr int msg_batch() { return NT == 1024 ? 1 : 2; }

// One trade by the whole CTA.  Returns false when a wait gave up.
template <int NT, class HT>
__device__ bool uni_trade(BlockTeam<NT>& tm, const UniCtx& c, int64_t k, const TradeWs<HT>& w, int hbits,
                          int32_t* hist, int64_t* s_sel, int* s_abort) {
  const int32_t u = c.tp[2 * k], v = c.tp[2 * k + 1];
  const int du = static_cast<int>(c.rp[u + 1] - c.rp[u]), dv = static_cast<int>(c.rp[v + 1] - c.rp[v]);
  const int32_t nu = c.nxt[2 * k], nv = c.nxt[2 * k + 1];
  const int E = du + dv;
  const int H = 1 << hbits;
  const int2* inu = c.inbox + c.ib[2 * k];
  const int2* inv = c.inbox + c.ib[2 * k + 1];
  // 1. gather both inboxes: plain L2 loads, and a bounded wait only for an
  //    entry still in flight; clear the hash
  bool ok = true;
#pragma unroll 4
  for (int e = tm.rank; e < E; e += NT) {
    const int side = e >= du;
    const int2* p = side ? inv + (e - du) : inu + e;
    int2 m = __ldcg(p);
    if (m.x == -1 && !wait_entry(p, c.err, c.wait_ns, &m)) {
      ok = false;
      m = make_int2(0, kInf);
    }
    w.ent[e] = m;
    w.flag[e] = static_cast<uint8_t>(side);
  }
  for (int s = tm.rank; s < H; s += NT) w.hash[s] = 0;
  if (!ok) atomicExch(s_abort, 1);
  tm.sync();
  if (*s_abort) return false;
  // 2. u's neighbours into the hash (entry index + 1)
  for (int e = tm.rank; e < du; e += NT) {
    uint32_t s = hash_slot(w.ent[e].x, hbits);
    while (atomicCAS(&w.hash[s], HT(0), static_cast<HT>(e + 1)) != HT(0)) s = (s + 1) & (H - 1);
  }
  tm.sync();
  // 3. v's neighbours look themselves up: common neighbours and the edge {u, v}
  for (int e = du + tm.rank; e < E; e += NT) {
    const int32_t x = w.ent[e].x;
    uint8_t f = 1;
    if (x == u) f |= 4;
    uint32_t s = hash_slot(x, hbits);
    for (;;) {
      const int32_t h = static_cast<int32_t>(w.hash[s]);
      if (h == 0) break;
      if (w.ent[h - 1].x == x) {
        f |= 2;
        w.flag[h - 1] = 2;   // side 0, common
        break;
      }
      s = (s + 1) & (H - 1);
    }
    w.flag[e] = f;
  }
  tm.sync();
  // 4. D = the rest, keyed by trade k's shuffle keys (Philox on (node id, k))
  const uint64_t gi = c.first + static_cast<uint64_t>(k);
  int64_t cnt = 0;
#pragma unroll 4
  for (int e = tm.rank; e < E; e += NT) {
    uint8_t f = w.flag[e];
    if (f == 0 && w.ent[e].x == v) w.flag[e] = f = 4;
    if ((f & 6) == 0) {
      const uint32_t id = static_cast<uint32_t>(c.order[w.ent[e].x]);
      const Philox4 r = philox4x32_10(id, static_cast<uint32_t>(gi), static_cast<uint32_t>(gi >> 32), 6u, c.seed);
      w.key[e] = (static_cast<uint64_t>(r.w0) << 32) | r.w1;
      cnt += 1 + ((f & 1) ? 0 : (int64_t(1) << 32));
    }
  }
  cnt = tm.sum(cnt);
  const int nd = static_cast<int>(cnt & 0xffffffff), na = static_cast<int>(cnt >> 32);
  // 5. sigma(D) sorts D by (key, node id); u receives the first na (Fig. 2).
  //    Radix select of the na-th smallest key, 8 bits at a time from the top.
  uint64_t prefix = 0, mask = 0;
  int r = na;
  bool tie = false;
  if (na > 0 && na < nd) {
    for (int shift = 56;; shift -= 8) {
      for (int b = tm.rank; b < 256; b += NT) hist[b] = 0;
      tm.sync();
#pragma unroll 4
      for (int e = tm.rank; e < E; e += NT)
        if ((w.flag[e] & 6) == 0 && (w.key[e] & mask) == prefix) atomicAdd(&hist[(w.key[e] >> shift) & 255], 1);
      tm.sync();
      const int hb = tm.rank < 256 ? hist[tm.rank] : 0;
      const int64_t below = tm.exscan(hb);
      if (tm.rank < 256 && below < r && r <= below + hb) {
        s_sel[0] = tm.rank;
        s_sel[1] = hb;
        s_sel[2] = below;
      }
      tm.sync();
      const int b = static_cast<int>(s_sel[0]), size = static_cast<int>(s_sel[1]);
      r -= static_cast<int>(s_sel[2]);
      prefix |= static_cast<uint64_t>(b) << shift;
      mask |= uint64_t(255) << shift;
      if (size == 1) break;
      if (shift == 0) {
        tie = true;   // several elements share the full key: node id decides
        break;
      }
    }
  }
  // decision: below the threshold's bucket to u, above to v, within it by rank
  int moved = 0;
#pragma unroll 2
  for (int e = tm.rank; e < E; e += NT) {
    const uint8_t f = w.flag[e];
    if (f & 6) continue;
    bool to_u;
    if (na == 0) to_u = false;
    else if (na == nd) to_u = true;
    else {
      const uint64_t km = w.key[e] & mask;
      if (km != prefix) to_u = km < prefix;
      else if (!tie) to_u = r >= 1;   // the single element of the last bucket is the na-th
      else {
        to_u = tied_before(c, w.ent, w.key, w.flag, E, e) < r;
      }
    }
    if (to_u) w.flag[e] = f | 8;
    moved += to_u == ((f & 1) != 0);   // an edge end that changes node
  }
  if (c.swaps) {
    if (moved) atomicAdd(&c.swaps[0], static_cast<unsigned long long>(moved));
    if (tm.rank == 0) atomicAdd(&c.swaps[1], static_cast<unsigned long long>(E));
  }
  tm.sync();
  // 6. every resulting edge goes on: common neighbours and the edge {u, v}
  //    stay, D as decided; atomics of a thread's messages overlap in batches
  for (int e0 = 0; e0 < E; e0 += NT * msg_batch<NT>()) {
    Msg m[msg_batch<NT>()];
    bool has[msg_batch<NT>()];
#pragma unroll
    for (int j = 0; j < msg_batch<NT>(); ++j) {
      const int e = e0 + j * NT + tm.rank;
      has[j] = false;
      if (e < E) {
        const uint8_t f = w.flag[e];
        const int2 en = w.ent[e];
        if (f & 4) {
          if (!(f & 1)) {   // the edge {u, v}: from u's entry only
            m[j] = {u, nu, v, nv, 0, 0ull};
            has[j] = true;
          }
        } else {
          const bool at_u = (f & 2) ? !(f & 1) : ((f & 8) != 0);
          m[j] = {at_u ? u : v, at_u ? nu : nv, en.x, en.y, 0, 0ull};
          has[j] = true;
        }
        if (has[j]) reserve(c, m[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < msg_batch<NT>(); ++j)
      if (has[j]) deliver(c, m[j]);
  }
  tm.sync();   // the work space is reused by the next trade
  return true;
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) k_uni_exec(UniCtx c) {
  extern __shared__ __align__(16) char usm[];
  __shared__ int64_t red[BlockTeam<NT>::kRedSlots];
  __shared__ int32_t hist[256];
  __shared__ int64_t s_sel[3];
  __shared__ int64_t s_k;
  __shared__ int s_abort;
  BlockTeam<NT> tm(red);
  if (threadIdx.x == 0) s_abort = 0;
  const TradeWs ws_smem = carve_ws(usm, uni_smem_elems<NT>());
  const TradeWs ws_glob =
      c.gslice ? carve_ws(c.gslice + static_cast<size_t>(blockIdx.x) * c.slice_elems * kWsBytesPerElem, c.slice_elems)
               : ws_smem;
  for (;;) {
    if (threadIdx.x == 0) s_k = take_ticket(c);
    tm.sync();
    const int64_t k = s_k;
    if (k < 0) break;
    const int32_t u = c.tp[2 * k], v = c.tp[2 * k + 1];
    const int64_t du = c.rp[u + 1] - c.rp[u];
    const int64_t E = du + (c.rp[v + 1] - c.rp[v]);
    bool ok;
    if (E <= uni_smem_elems<NT>()) {
      ok = uni_trade(tm, c, k, ws_smem, hash_bits(2 * du), hist, s_sel, &s_abort);
    } else if (du <= kHash16MaxDu) {
      TradeWs<uint16_t> w16{ws_glob.ent, ws_glob.key, reinterpret_cast<uint16_t*>(usm), ws_glob.flag};
      ok = uni_trade(tm, c, k, w16, hash_bits((4 * du + 2) / 3), hist, s_sel, &s_abort);
    } else {
      ok = uni_trade(tm, c, k, ws_glob, hash_bits(2 * du), hist, s_sel, &s_abort);
    }
    if (!ok) {
      if (threadIdx.x == 0) latch(c.err, kErrUniformWait);
      break;
    }
  }
}

// Every output row full.
// Every output row full, and every trade queued and taken exactly once.
__global__ void k_uni_check(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ocur,
                            const unsigned long long* __restrict__ ctr, int64_t L, int32_t* err) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long l = static_cast<unsigned long long>(L);
    if (ctr[kTail] != l) latch(err, kErrUniform);
  }
  for (int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; x < n; x += int64_t(gridDim.x) * blockDim.x)
    if (ocur[x] != rp[x + 1] - rp[x]) latch(err, kErrRowLength);
}

unsigned grid_for_work(int64_t work, int num_sms) {
  const int64_t want = (work + 255) / 256;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(num_sms) * 16)));
}

template <class T>
cudaError_t grow(Graph* h, T** p, int64_t count, size_t* bytes) {
  if (count <= 0) count = 1;
  void* q = nullptr;
  const cudaError_t e = dev_alloc(h, &q, sizeof(T) * static_cast<size_t>(count));
  if (e == cudaSuccess) {
    *p = static_cast<T*>(q);
    *bytes += sizeof(T) * static_cast<size_t>(count);
  }
  return e;
}

int uni_buffers(Graph* h, int64_t L) {
  UniBufs* b = h->uni;
  if (b && b->cap_trades >= L && b->n == h->n) return CB_OK;
  free_uniform(h);
  b = new UniBufs;
  h->uni = b;
  const int64_t n = h->n;
  b->cap_trades = L;
  b->n = n;
  size_t* by = &b->bytes;
  if (grow(h, &b->tp, 2 * L, by) || grow(h, &b->dslot, 2 * L, by) || grow(h, &b->ib, 2 * L + 1, by) ||
      grow(h, &b->suc, 2 * L, by) || grow(h, &b->nxt, 2 * L, by) || grow(h, &b->fill, L, by) ||
      grow(h, &b->queue, L, by) || grow(h, &b->occ, n, by) || grow(h, &b->sbeg, n + 1, by) ||
      grow(h, &b->ocur, n, by) || grow(h, &b->ctr, kCtrWords, by))
    return fail(h, CB_ENOMEM, "device allocation failed (uniform trades)");
  const size_t ws = std::max(scan_ws_bytes(n), scan_ws_bytes(2 * L));
  void* q = nullptr;
  if (dev_alloc(h, &q, ws)) return fail(h, CB_ENOMEM, "device allocation failed (uniform trades)");
  b->scan_ws = q;
  b->bytes += ws;
  return CB_OK;
}

}  // namespace

void free_uniform(Graph* h) {
  UniBufs* b = h->uni;
  if (!b) return;
  void* bufs[] = {b->tp, b->dslot, b->ib, b->suc, b->nxt, b->fill, b->queue, b->occ, b->sbeg, b->ocur, b->ctr,
                  b->scan_ws};
  if (h->stream) {
    for (void* p : bufs)
      if (p) cudaFreeAsync(p, h->stream);
    if (b->inbox) cudaFreeAsync(b->inbox, h->stream);
    if (b->gslice) cudaFreeAsync(b->gslice, h->stream);
  }
  h->dev_bytes -= static_cast<int64_t>(b->bytes + b->inbox_bytes + b->slice_bytes);
  delete b;
  h->uni = nullptr;
}

int uniform_trades(Graph* h, uint64_t count) {
  if (h->nseg != 1) return fail(h, CB_EINVAL, "uniform trades are for handles of one graph");
  const int64_t n = h->n;
  if (n < 2 || count == 0) {
    h->uni_next += count;
    return CB_OK;
  }
  cudaStream_t s = h->stream;
  const int64_t launches0 = h->launches;
  const int64_t chunk = std::max<int64_t>(n / 2, kUniChunkMin);
  int rc;
  if ((rc = uni_buffers(h, std::min<int64_t>(chunk, static_cast<int64_t>(std::min<uint64_t>(count, 1ull << 40))))))
    return rc;
  UniBufs* b = h->uni;
  // kernel resources: occupancy of the persistent executor, its sort space
  const int NT = h->uni_threads;
  const void* exec = NT == 1024 ? reinterpret_cast<const void*>(k_uni_exec<1024>)
                     : NT == 512 ? reinterpret_cast<const void*>(k_uni_exec<512>)
                                 : reinterpret_cast<const void*>(k_uni_exec<256>);
  const int smem_elems = NT == 1024 ? uni_smem_elems<1024>() : uni_smem_elems<256>();
  const size_t smem = kWsBytesPerElem * smem_elems;
  CB_CUDA(h, cudaFuncSetAttribute(exec, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  int per_sm = 0;
  CB_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, exec, NT, smem));
  const int ctas = std::max(1, per_sm) * h->num_sms;
  const int64_t big = next_pow2_host(std::max<int64_t>(2 * h->maxdeg, 1));
  if (2 * h->maxdeg > smem_elems && (!b->gslice || b->slice_elems < big || b->ctas < ctas)) {
    if (b->gslice) {
      cudaFreeAsync(b->gslice, s);
      h->dev_bytes -= static_cast<int64_t>(b->slice_bytes);
      b->gslice = nullptr;
      b->slice_bytes = 0;
    }
    const size_t bytes = static_cast<size_t>(big) * kWsBytesPerElem * ctas;
    void* q = nullptr;
    if (dev_alloc(h, &q, bytes)) return fail(h, CB_ENOMEM, "device allocation failed (uniform sort space)");
    b->gslice = static_cast<char*>(q);
    b->slice_elems = big;
    b->slice_bytes = bytes;
    b->ctas = ctas;
  }
  // node id -> position of the current step
  if ((rc = invert_permutation(h, h->order[h->cur], h->pos_next))) return rc;
  const unsigned g1 = grid_for_work(n, h->num_sms);
  uint64_t done = 0;
  while (done < count) {
    const int64_t L = static_cast<int64_t>(std::min<uint64_t>(count - done, static_cast<uint64_t>(b->cap_trades)));
    const uint64_t first = h->uni_next + done;
    const unsigned gL = grid_for_work(L, h->num_sms);
    // the sequence in positions, its Suc lists and every slot's next trade
    k_uni_draw<<<gL, 256, 0, s>>>(L, first, h->seed, n, h->pos_next, h->rp[h->cur], b->tp, b->dslot);
    CB_CUDA(h, cudaGetLastError());
    CB_CUDA(h, cudaMemsetAsync(b->occ, 0, sizeof(int32_t) * n, s));
    k_uni_count<<<gL, 256, 0, s>>>(L, n, b->tp, b->occ, h->err);
    CB_CUDA(h, cudaGetLastError());
    CB_CUDA(h, exclusive_scan_i32(b->occ, b->sbeg, n, b->scan_ws, s, &h->launches));
    CB_CUDA(h, cudaMemsetAsync(b->occ, 0, sizeof(int32_t) * n, s));
    k_uni_fill<<<grid_for_work(2 * L, h->num_sms), 256, 0, s>>>(2 * L, b->tp, b->sbeg, b->occ, b->suc);
    CB_CUDA(h, cudaGetLastError());
    k_uni_sort<<<g1, 256, 0, s>>>(n, b->sbeg, b->suc, b->nxt);
    CB_CUDA(h, cudaGetLastError());
    CB_CUDA(h, exclusive_scan_i32(b->dslot, b->ib, 2 * L, b->scan_ws, s, &h->launches));
    int64_t total = 0;
    CB_CUDA(h, cudaMemcpyAsync(&total, b->ib + 2 * L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CB_CUDA(h, cudaStreamSynchronize(s));
    if (total > b->inbox_cap) {
      if (b->inbox) {
        cudaFreeAsync(b->inbox, s);
        h->dev_bytes -= static_cast<int64_t>(b->inbox_bytes);
        b->inbox = nullptr;
        b->inbox_cap = 0;
        b->inbox_bytes = 0;
      }
      const int64_t cap = total + total / 8 + 1024;
      void* q = nullptr;
      if (dev_alloc(h, &q, sizeof(int2) * static_cast<size_t>(cap)))
        return fail(h, CB_ENOMEM, "device allocation failed (uniform inboxes)");
      b->inbox = static_cast<int2*>(q);
      b->inbox_cap = cap;
      b->inbox_bytes = sizeof(int2) * static_cast<size_t>(cap);
    }
    // empty inboxes (every byte 0xff: node -1), counts, queue, output cursors
    if (total) CB_CUDA(h, cudaMemsetAsync(b->inbox, 0xff, sizeof(int2) * static_cast<size_t>(total), s));
    CB_CUDA(h, cudaMemsetAsync(b->fill, 0, sizeof(unsigned long long) * L, s));
    CB_CUDA(h, cudaMemsetAsync(b->queue, 0xff, sizeof(int32_t) * L, s));
    CB_CUDA(h, cudaMemsetAsync(b->ctr, 0, sizeof(unsigned long long) * kCtrWords, s));
    CB_CUDA(h, cudaMemsetAsync(b->ocur, 0, sizeof(int32_t) * n, s));
    const int spare = 1 - h->cur;
    UniCtx c;
    c.L = L;
    c.first = first;
    c.seed = h->seed;
    c.rp = h->rp[h->cur];
    c.order = h->order[h->cur];
    c.tp = b->tp;
    c.nxt = b->nxt;
    c.ib = b->ib;
    c.sbeg = b->sbeg;
    c.suc = b->suc;
    c.inbox = b->inbox;
    c.fill = b->fill;
    c.queue = b->queue;
    c.ctr = b->ctr;
    c.ocur = b->ocur;
    c.col_out = h->col[spare];
    c.wait_ns = h->uni_wait_ns;
    c.hold_trade = h->hold_trade;
    c.err = h->err;
    c.gslice = b->gslice;
    c.slice_elems = b->slice_elems;
    c.swaps = h->swap_stats ? reinterpret_cast<unsigned long long*>(h->swaps) : nullptr;
    k_uni_route<<<grid_for_work(n * 32, h->num_sms), 256, 0, s>>>(c, n, h->col[h->cur]);
    CB_CUDA(h, cudaGetLastError());
    if (NT == 1024) k_uni_exec<1024><<<ctas, 1024, smem, s>>>(c);
    else if (NT == 512) k_uni_exec<512><<<ctas, 512, smem, s>>>(c);
    else k_uni_exec<256><<<ctas, 256, smem, s>>>(c);
    CB_CUDA(h, cudaGetLastError());
    k_uni_check<<<g1, 256, 0, s>>>(n, c.rp, b->ocur, b->ctr, L, h->err);
    CB_CUDA(h, cudaGetLastError());
    h->launches += 7;
    if ((rc = check_device_error(h))) return rc;
    std::swap(h->col[h->cur], h->col[spare]);
    done += static_cast<uint64_t>(L);
  }
  h->uni_next += count;
  h->stats[5] = h->launches - launches0;
  // the recorded super steps name the old adjacency buffers; exports are stale
  drop_step_graphs(h);
  h->pairs_step = ~0ull;
  return CB_OK;
}

}  // namespace cb

extern "C" int cb_uniform_trades(cb_handle h, uint64_t count) {
  using namespace cb;
  if (!h) return fail(nullptr, CB_EINVAL, "NULL handle");
  if (h->latched) return fail(h, h->latched, "handle has a latched error: " + h->last_error);
  return uniform_trades(h, count);
}

extern "C" int cb_uniform_next(cb_handle h, uint64_t* next) {
  using namespace cb;
  if (!h || !next) return fail(h, CB_EINVAL, "bad argument");
  *next = h->uni_next;
  return CB_OK;
}

extern "C" int cb_uniform_pairs(uint64_t seed, int64_t n, uint64_t first, int64_t count, int32_t* pairs,
                                void* cuda_stream) {
  using namespace cb;
  if (n < 2 || n > 0x7fffffffLL || count < 0 || (count > 0 && !pairs))
    return fail(nullptr, CB_EINVAL, "cb_uniform_pairs: needs 2 <= n < 2^31, count >= 0 and a buffer");
  if (count == 0) return CB_OK;
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_uni_draw<<<grid_for_work(count, num_sms), 256, 0, s>>>(count, first, seed, n, nullptr, nullptr, pairs, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "k_uni_draw");
  return CB_OK;
}

extern "C" int cb_successors(int64_t n, const int32_t* pairs, int64_t count, int64_t* suc_begin, int32_t* suc,
                             void* cuda_stream) {
  using namespace cb;
  if (n < 0 || n > 0x7fffffffLL || count < 0 || count > 0x3fffffffLL || !suc_begin || (count > 0 && (!pairs || !suc)))
    return fail(nullptr, CB_EINVAL, "cb_successors: bad n, count or buffer");
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // scratch: occurrence counts / cursors, slot lists, an error word, scan space
  const size_t ws = scan_ws_bytes(n);
  const size_t bytes = sizeof(int32_t) * (static_cast<size_t>(n) + 2 * static_cast<size_t>(count) + 1) + ws + 16;
  char* scratch = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaMallocAsync");
  int32_t* occ = reinterpret_cast<int32_t*>(scratch);
  int32_t* slots = occ + n;
  int32_t* err = slots + 2 * count;
  void* scan = scratch + ((sizeof(int32_t) * (n + 2 * count + 1) + 15) & ~size_t(15));
  int rc = CB_OK;
  int32_t herr = 0;
  const unsigned g = grid_for_work(std::max<int64_t>(n, 2 * count), num_sms);
  if ((e = cudaMemsetAsync(occ, 0, sizeof(int32_t) * (n + 2 * count + 1), s)) != cudaSuccess) goto cuda_error;
  if (count) {
    k_uni_count<<<g, 256, 0, s>>>(count, n, pairs, occ, err);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_error;
  }
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) goto cuda_error;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_error;
  if (herr) {
    rc = fail(nullptr, CB_EINVAL, "cb_successors: a node outside [0, n) or a pair of equal nodes");
    goto done;
  }
  if ((e = exclusive_scan_i32(occ, suc_begin, n, scan, s)) != cudaSuccess) goto cuda_error;
  if (count) {
    if ((e = cudaMemsetAsync(occ, 0, sizeof(int32_t) * n, s)) != cudaSuccess) goto cuda_error;
    k_uni_fill<<<g, 256, 0, s>>>(2 * count, pairs, suc_begin, occ, slots);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_error;
    k_uni_sort<<<g, 256, 0, s>>>(n, suc_begin, slots, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_error;
    k_uni_trade_index<<<g, 256, 0, s>>>(2 * count, slots, suc);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_error;
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto cuda_error;
  goto done;
cuda_error:
  rc = cuda_fail(nullptr, e, "cb_successors");
done:
  cudaFreeAsync(scratch, s);
  return rc;
}
