// Internal state and helpers of libcb (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "cb.h"

namespace cb {

// Device-side error codes latched in Graph::err (first one wins).
enum DevErr : int32_t {
  kErrNone = 0,
  kErrRowLength = 1,     // a rebuilt row does not match the degree
  kErrRowSide = 2,       // entry written to the wrong row of a trade
  kErrValidate = 3,      // input graph not simple / symmetric / in range
  kErrBucket = 4,        // permutation bucket bookkeeping failed
  kErrResolve = 5,       // a dependency wait of the in-order pass gave up
  kErrStage = 6,         // a bulk copy into shared memory did not complete in time
  kErrUniform = 7,       // uniform trades: an inbox or the run queue overflowed, or a message missed its trade
  kErrUniformWait = 8,   // uniform trades: a wait for a queued trade or an inbox entry gave up
};
// The codes that report a bounded wait running out (CB_ETIMEOUT).
inline bool is_timeout(int32_t e) { return e == kErrResolve || e == kErrStage || e == kErrUniformWait; }

struct UniBufs;        // uniform-trade buffers (uniform.cu)
struct PresenceBufs;   // edge presence record (autocorr.cu)

constexpr int kBucketCapMax = 4096;  // largest "bucket_cap"
constexpr int kTileMaxCap = 128;    // largest trade (deg u + deg v) on the flat tile path
constexpr int kBlockMaxCap = 2048;  // largest trade on the 256-thread path
constexpr int kBlockMaxDefault = 1024;   // default of the "block_max" option
constexpr int kSmemMaxCap = 8192;   // largest trade kept in shared memory on the 1024-thread path
constexpr int kBlockThreads = 256;  // CTA size of the block path
constexpr int kCounters = 96;       // device counters per handle
// Trade size classes of the threshold phase (one team size each) and the
// device counters of a super step.
constexpr int kClasses = 9;
constexpr int kWarpClasses = 3;     // classes 0..2 run on warps or parts of a warp
constexpr int kCtrClsLen = 0;       // [0, kClasses): trades per class
constexpr int kCtrClsStart = 10;    // [10, 10 + kClasses): first entry of each class in the class lists
constexpr int kCtrClaims = 19;      // chunks claimed by the in-order pass
constexpr int kCtrFirstLen = 20;    // [20, 20 + kClasses): trades per class in the first pass
constexpr int kCtrFirstEnt = 29;    // [29, 29 + kClasses): directed entries per class in the first pass
constexpr int kCtrPassLeft = 40;    // [40, 40 + kRetryPassesMax + 2): trades left deferred after pass r
constexpr int kRetryPassesMax = 4;
constexpr int kCtrPassSmall = 48;   // [48, 54): of those, the small ones (listed from the front of the list)
constexpr int kCtrPassBig = 56;     // [56, 62): the others (listed from the back)
constexpr int kCtrListClaim = 64;   // [64, 64 + 3 kRetryPassesMax]: list positions claimed by the passes' kernels
constexpr int kCtrListOk = 80;      // 1: the in-order pass runs on the sorted list of the last pass
constexpr int kCtrListN = 81;       // the sorted list's length
static_assert(40 + kRetryPassesMax + 2 <= 48 && 64 + 3 * kRetryPassesMax < 80, "counter layout");
constexpr int kStats = 7 + 2 * kClasses;   // counters cb_stats reports
constexpr int kTimings = 6 + kClasses;     // values cb_timings reports
constexpr int kCtrGws = kCounters - 1;   // trades whose workspace is in global memory
constexpr int kMaxLcgGaps = 1024;   // p - n for the relaxed permutation (prime gaps below 2^31 are far smaller)

// One independent graph of a handle.  A plain handle holds one; a batch handle
// holds many side by side: graph i owns node ids and positions [off, off+span),
// and its keys use local ids and positions with its own seed and step, so it
// evolves exactly as it would alone.  An odd graph in a batch gets one padding
// node of degree 0 whose permutation key is the largest possible: it always
// takes the last position, and its trade with the node before it changes
// nothing, which is the untraded last position of an odd graph.
struct Seg {
  uint64_t seed;
  int64_t off;           // first node id (= first position)
  int64_t n;             // real nodes
  int64_t span;          // n, or n + 1 with a padding node
  int64_t bucket_base;   // first permutation bucket
  int64_t m;             // undirected edges
  int64_t pair_off;      // first exported pair
  uint32_t g;            // super step (advanced on the device at the end of each step)
  int32_t B;             // permutation bucket bits
};

struct Graph {
  int64_t n = 0, nnz = 0, m = 0, T = 0, ntasks = 0;
  uint64_t seed = 0, g = 0;
  // segments (graphs) of the handle
  int nseg = 1;
  Seg* segs = nullptr;            // device table (nseg)
  int32_t* seg_of = nullptr;      // device: segment of each node id / position (null when nseg == 1)
  Seg* hsegs = nullptr;           // host copy (g not kept current)
  int64_t nbuckets = 1;           // permutation buckets over all segments
  int32_t* pairs = nullptr;       // batch export: every graph's pairs, local ids
  uint64_t pairs_step = ~0ull;    // super step the pairs were exported at
  // CUDA graph of one super step per ping-pong parity
  bool use_graph = false;
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  int64_t step_launches = 0;      // kernels in one captured super step
  int64_t maxdeg = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, num_sms = 0;

  // constant per graph
  int32_t* deg_id = nullptr;      // degree by node id
  int64_t* rp_id = nullptr;       // id-space row offsets (n+1)
  // per super step (ping-pong index `cur`)
  int cur = 0;
  int32_t* order[2] = {nullptr, nullptr};  // node at each position
  int64_t* rp[2] = {nullptr, nullptr};     // position-space row offsets (n+1)
  int32_t* col[2] = {nullptr, nullptr};    // position-space rows, ascending
  int32_t* pos_next = nullptr;             // position of each node id in step g+1
  int32_t* M = nullptr;                    // step-g position -> step-(g+1) position
  int32_t* Minv = nullptr;                 // step-(g+1) position -> step-g position
  int32_t* deg_next = nullptr;             // degree by step-(g+1) position
  uint16_t* stash = nullptr;               // per placed entry (step g+1 layout): bit0 own flip, bits 1.. far key prefix
  uint64_t* thr_key = nullptr;             // per trade: threshold key
  uint8_t* thr_top = nullptr;              // per trade: top 6 bits of the threshold key
  uint64_t* thr_tb = nullptr;              // per trade: threshold tie-break (lo<<32|hi)
  uint32_t* done = nullptr;                // per trade: 1 once the threshold is published (cleared per step)
  int4* far_pack = nullptr;                // per trade: new positions of its nodes, threshold prefix (rebuild)
  int32_t* lists = nullptr;                // trades of every size class, class after class, index order within
  int32_t* dlist = nullptr;                // 2 ntasks: the trades each pass deferred, for the next one
  int32_t* cls_flag = nullptr;             // scratch: per-chunk class counts, then the rebuild's chunk rows
  int64_t* cls_scan = nullptr;             // scratch: their exclusive scan
  int64_t* counters = nullptr;             // list lengths, deferred count, claims (kCounters)
  int32_t* err = nullptr;                  // latched device error
  // workspaces
  void* ws_global = nullptr;               // global workspace for trades too big for smem
  size_t ws_slice = 0;                     // bytes per CTA slice
  int ws_ctas = 0;                         // number of slices
  void* sort_ws = nullptr;                 // permutation sort scratch
  size_t sort_ws_bytes = 0;
  void* scan_ws = nullptr;
  size_t scan_ws_bytes = 0;
  int64_t* host_counters = nullptr;        // host mirror of counters
  int64_t dev_bytes = 0, dev_bytes_peak = 0;   // device memory held by the handle

  // knobs
  int tile_max = kTileMaxCap;
  int tile_paths = 1;   // threshold phase of small trades: 1 one warp per trade, 0 256-thread CTAs
  int fix_passes = 0;   // passes of the rebuild's fix-up over slices of the far trades (0: sized for L2)
  int cta_paths = 1;    // threshold phase of larger trades: 1 register-resident CTA kernels, 0 shared-memory ones
  int cand_max = 32;    // register paths: candidates ranked directly (tests lower it to force radix digits)
  uint64_t wait_ns = 1000000000ull;       // longest single wait of a super step (dependency, bulk copy)
  uint64_t uni_wait_ns = 20000000000ull;  // longest single wait of the uniform-trade executor
  int hold_publish = 0;                   // test hook: trades never publish their done flags
  int64_t hold_trade = -1;                // test hook: uniform trade whose messages are dropped
  int block_max = kBlockMaxDefault;
  int smem_max = kSmemMaxCap;
  int bucket_cap = 2048;
  int inorder_threads = 1024;   // CTA size of the in-order threshold pass (256 or 1024)
  int retry_passes = 2;         // parallel passes over the deferred trades before the in-order pass
  int lane_teams = 1;           // trades up to 32 / 64 entries on teams of 8 / 16 lanes
  int uni_threads = 1024;       // CTA size of the uniform-trade executor (256, 512 or 1024)
  bool wide_pack = false;       // 16-byte far-trade records even when 8 bytes would do (tests)
  // relaxed global trade: permutations from h(x) = (a x + b) mod p
  bool relaxed = false;
  uint64_t lcg_p = 0;           // smallest prime >= n
  uint64_t* lcg_ab = nullptr;   // device: a, b of the step being prepared
  int64_t* lcg_gaps = nullptr;  // device: gap count, then the sorted gap values

  // uniform single trades (uniform.cu)
  UniBufs* uni = nullptr;
  uint64_t uni_next = 0;        // index of the next uniform trade
  // edge presence record for the autocorrelation of Section 5.1 (autocorr.cu)
  PresenceBufs* pres = nullptr;
  // swap counts (swaps.cu): device pair (performed, possible), when on
  bool swap_stats = false;
  int64_t* swaps = nullptr;

  // stats of the last cb_global_trades
  int64_t stats[kStats] = {0};
  int64_t launches = 0;                    // kernel launches issued by this handle
  bool timing = false;                     // record CUDA events around the phases
  // events, in two sets that super steps use in turn (the host waits for a
  // step's events only when the set comes round again, two steps later):
  // [0..4) phase bounds, [4, 4 + kClasses + 1) bounds of the first pass's
  // class kernels, then the end of the retry passes
  cudaEvent_t ev[2][4 + kClasses + 2] = {};
  int ev_set = 0;                          // the set the next super step records
  bool ev_pending[2] = {false, false};     // recorded, not yet added to phase_ms
  // permutation+prep, thresholds, rebuild, whole step, the first pass's
  // kernel of each size class, the retry passes, the in-order pass
  double phase_ms[kTimings] = {};
  int latched = CB_OK;
  std::string last_error;
};

inline int64_t next_pow2_host(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Records an error on the graph (or globally) and returns the code.
int fail(Graph* g, int code, const std::string& msg);
int cuda_fail(Graph* g, cudaError_t e, const char* what);

#define CB_CUDA(g, call)                                        \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::cb::cuda_fail((g), e_, #call); \
  } while (0)

// ---- kernels / host launchers implemented in the .cu files ----
// scan.cu
size_t scan_ws_bytes(int64_t n);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total
cudaError_t exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s,
                               int64_t* launches = nullptr);

// permute.cu
size_t perm_ws_bytes(int64_t n, int64_t nbuckets);
int bucket_bits(int64_t n);
// order_out[p] = node at position p; pos_out[x] = position of x (may be null).
// Each segment uses its device step counter + dg, or the step g_abs for all
// when g_abs >= 0.
int compute_permutation(Graph* h, uint32_t dg, int64_t g_abs, int32_t* order_out, int32_t* pos_out);
// M, deg_next and rp[1-cur] for the step after the current one
int prepare_next(Graph* h);

// rows.cu
// dst row q <- src row rowmap[q] with values mapped through valmap (identity if null), ascending
int permute_rows(Graph* h, int64_t nrows, const int64_t* src_rp, const int32_t* src_col,
                 const int32_t* rowmap, const int32_t* valmap, const int64_t* dst_rp, int32_t* dst_col);
// simple and symmetric, or kErrValidate latched; `grouped` is scratch of
// row_ptr[n] int32 (not synchronising)
int validate_sorted_graph(Graph* h, const int64_t* rp, const int32_t* col, int64_t n, int32_t* grouped);
// *sorted = every row strictly increasing (synchronises)
int rows_sorted(Graph* h, const int64_t* rp, const int32_t* col, int64_t n, bool* sorted);
// like permute_rows without sorting (rows keep their order)
int relabel_rows(Graph* h, int64_t nrows, const int64_t* src_rp, const int32_t* src_col, const int32_t* rowmap,
                 const int32_t* valmap, const int64_t* dst_rp, int32_t* dst_col);
int check_row_offsets(Graph* h, const int64_t* rp, int64_t n);
int invert_permutation(Graph* h, const int32_t* order, int32_t* pos);
// canonical pairs (x < y, sorted, local ids) of the current step into `pairs`
// (2m int32, device); uses the spare adjacency buffer
int export_sorted_pairs(Graph* h, int32_t* pairs);

// trade.cu
int super_step(Graph* h);
int flush_timing(Graph* h, int set, bool add);   // wait for a recorded event set; add it to phase_ms
int init_trade_kernels(Graph* h);   // one-time kernel attributes (outside stream capture)
int init_perm_kernels(Graph* h);
size_t trade_ws_slice_bytes(int64_t max_trade);

// api.cu
// stream-ordered device allocation counted in the handle's device bytes
cudaError_t dev_alloc(Graph* h, void** p, size_t bytes);
// read the latched device error word (synchronises the stream)
int check_device_error(Graph* h);
// forget the recorded super-step graphs (they are recorded again when next needed)
void drop_step_graphs(Graph* h);

// swaps.cu
int count_swaps(Graph* h);                 // add the last super step's counts
int set_swap_stats(Graph* h, bool on);     // on: counts from zero

// uniform.cu
int uniform_trades(Graph* h, uint64_t count);
void free_uniform(Graph* h);

// autocorr.cu
int set_presence(Graph* h, int64_t T);   // T > 0: record the next T super steps (and now); 0: stop
int record_presence(Graph* h);           // the current state, while recording
void free_presence(Graph* h);

// device bytes a plain handle of n nodes / nnz entries / largest degree takes (upper estimate)
int64_t estimate_handle_bytes(int64_t n, int64_t nnz, int64_t maxdeg, int num_sms);
// record the CUDA graphs of the super step now (when the cuda_graph option is on)
int prepare_step_graphs(Graph* h);

}  // namespace cb

struct cb_graph : cb::Graph {};
