// The serving loop declared in include/cb_serve.h: requests admitted by a
// device-memory budget, resident on their own streams, stepped together.
//
// Two host threads share one mutex-protected table of requests:
//   admitter  queued -> resident (create the state, record its CUDA graphs)
//             finished -> done   (export the edges to host memory, release)
//   stepper   issues super steps round robin over the resident requests,
//             at most `depth` in flight each, tracked with CUDA events.
// A request's handle is used by one thread at a time: the admitter until it
// is handed to the stepper, the stepper until its last super step has
// completed, then the admitter again.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cb_internal.cuh"
#include "cb_serve.h"

namespace cb {
namespace {

constexpr int kMaxDepth = 8;

enum class St { Queued, Resident, Finished, Done };

struct Request {
  int64_t id = 0;
  int64_t n = 0, nnz = 0, maxdeg = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  uint64_t seed = 0;
  uint32_t steps = 0;
  int64_t est = 0;
  St st = St::Queued;
  cb_handle h = nullptr;
  cudaStream_t stream = nullptr;
  uint32_t issued = 0;
  cudaEvent_t ev[kMaxDepth] = {};
  uint32_t completed = 0;           // super steps known complete
  std::vector<int32_t> edges;
  int64_t m = 0;
  int rc = CB_OK;
  std::string err;
  double t[4] = {0, 0, 0, 0};       // submitted, admitted, resident, finished
};

struct Server {
  int64_t budget = 0;
  int max_active = 1, depth = 2, device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit, cv_step, cv_done;
  bool stop = false;
  int64_t next_id = 0;
  std::map<int64_t, std::shared_ptr<Request>> all;
  std::deque<std::shared_ptr<Request>> queue;       // waiting for admission, arrival order
  std::vector<std::shared_ptr<Request>> resident;   // owned by the stepper
  std::deque<std::shared_ptr<Request>> finished;    // steps complete, to export
  std::deque<int64_t> done_ids;                     // not yet returned by poll
  int64_t reserved = 0, reserved_peak = 0, steps_issued = 0, n_done = 0, n_failed = 0, n_submitted = 0;
  int n_resident = 0;
  std::thread admitter, stepper;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

void fail_request(Server*, const std::shared_ptr<Request>& r, int rc, const std::string& msg) {
  r->rc = rc;
  r->err = msg;
}

// Called with the lock held: the request is done (result ready or failed).
void mark_done(Server* S, const std::shared_ptr<Request>& r) {
  r->st = St::Done;
  r->t[3] = S->now();
  ++S->n_done;
  if (r->rc != CB_OK) ++S->n_failed;
  S->done_ids.push_back(r->id);
  S->cv_done.notify_all();
}

void release_request_device(Request* r) {
  for (auto& e : r->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (r->h) {
    cb_destroy(r->h);
    r->h = nullptr;
  }
  if (r->stream) {
    cudaStreamDestroy(r->stream);
    r->stream = nullptr;
  }
}

// Create the device state of an admitted request (no lock held).
void make_resident(Server* S, const std::shared_ptr<Request>& r) {
  cudaSetDevice(S->device);
  cudaError_t e = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking);
  for (int i = 0; i < S->depth && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&r->ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fail_request(S, r, CB_ECUDA, std::string("stream or event creation failed: ") + cudaGetErrorString(e));
    return;
  }
  int rc = cb_create(r->n, r->rp.data(), r->col.data(), r->seed, 0, CB_HOST, r->stream, &r->h);
  if (rc == CB_OK) rc = cb_set_option(r->h, "cuda_graph", 1);
  if (rc == CB_OK) rc = prepare_step_graphs(r->h);
  if (rc != CB_OK) {
    fail_request(S, r, rc, r->h ? cb_last_error(r->h) : cb_last_error(nullptr));
    return;
  }
  std::vector<int64_t>().swap(r->rp);   // the device holds the graph now
  std::vector<int32_t>().swap(r->col);
}

// Export the result of a request whose super steps are complete (no lock held).
void export_result(Server* S, const std::shared_ptr<Request>& r) {
  cudaSetDevice(S->device);
  int64_t m = 0;
  int rc = cb_export_edges(r->h, nullptr, 0, &m, CB_HOST);
  if (rc == CB_OK) {
    r->edges.resize(static_cast<size_t>(2 * m));
    rc = cb_export_edges(r->h, r->edges.data(), m, &m, CB_HOST);
  }
  if (rc == CB_OK) rc = cb_sync(r->h);
  if (rc != CB_OK) fail_request(S, r, rc, cb_last_error(r->h));
  r->m = m;
}

void admitter_loop(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    // finished requests first: they free memory
    if (!S->finished.empty()) {
      auto r = S->finished.front();
      S->finished.pop_front();
      lk.unlock();
      if (r->rc == CB_OK) export_result(S, r);
      release_request_device(r.get());
      lk.lock();
      S->reserved -= r->est;
      --S->n_resident;
      mark_done(S, r);
      continue;
    }
    // admit the head of the queue if it fits
    if (!S->queue.empty()) {
      auto r = S->queue.front();
      if (r->est > S->budget) {
        S->queue.pop_front();
        fail_request(S, r, CB_ENOMEM, "request needs more device memory than the whole budget");
        mark_done(S, r);
        continue;
      }
      if (S->n_resident < S->max_active && S->reserved + r->est <= S->budget) {
        S->queue.pop_front();
        S->reserved += r->est;
        S->reserved_peak = std::max(S->reserved_peak, S->reserved);
        ++S->n_resident;
        r->t[1] = S->now();
        lk.unlock();
        make_resident(S, r);
        lk.lock();
        r->t[2] = S->now();
        if (r->rc != CB_OK) {
          lk.unlock();
          release_request_device(r.get());
          lk.lock();
          S->reserved -= r->est;
          --S->n_resident;
          mark_done(S, r);
        } else {
          r->st = St::Resident;
          S->resident.push_back(r);
          S->cv_step.notify_all();
        }
        continue;
      }
    }
    S->cv_admit.wait_for(lk, std::chrono::milliseconds(50));
  }
}

void stepper_loop(Server* S) {
  cudaSetDevice(S->device);
  std::vector<std::shared_ptr<Request>> mine;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) return;
      // take over newly resident requests
      for (auto& r : S->resident) mine.push_back(r);
      S->resident.clear();
      if (mine.empty()) {
        S->cv_step.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
    }
    bool progress = false;
    for (size_t i = 0; i < mine.size();) {
      auto& r = mine[i];
      // retire completed super steps (events complete in issue order)
      while (r->completed < r->issued &&
             cudaEventQuery(r->ev[r->completed % S->depth]) == cudaSuccess) {
        ++r->completed;
        progress = true;
      }
      if (r->rc == CB_OK && r->issued < r->steps && r->issued - r->completed < static_cast<uint32_t>(S->depth)) {
        int rc = cb_global_trades(r->h, 1);
        if (rc == CB_OK && cudaEventRecord(r->ev[r->issued % S->depth], r->stream) != cudaSuccess) rc = CB_ECUDA;
        if (rc != CB_OK) {
          fail_request(S, r, rc, cb_last_error(r->h));
        } else {
          ++r->issued;
          progress = true;
          std::lock_guard<std::mutex> lk(S->mu);
          ++S->steps_issued;
        }
      }
      if (r->rc != CB_OK || r->completed == r->steps) {
        std::lock_guard<std::mutex> lk(S->mu);
        r->st = St::Finished;
        S->finished.push_back(r);
        S->cv_admit.notify_all();
        mine.erase(mine.begin() + static_cast<std::ptrdiff_t>(i));
        progress = true;
        continue;
      }
      ++i;
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace
}  // namespace cb

struct cb_server : cb::Server {};

using namespace cb;

extern "C" {

int cb_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t depth, cb_server_t* out) {
  if (!out || hbm_budget_bytes <= 0 || max_active < 1 || depth < 1 || depth > kMaxDepth)
    return fail(nullptr, CB_EINVAL, "cb_server_create: bad budget, max_active or depth");
  *out = nullptr;
  cb_server* S = new (std::nothrow) cb_server();
  if (!S) return fail(nullptr, CB_ENOMEM, "host allocation failed");
  S->budget = hbm_budget_bytes;
  S->max_active = max_active;
  S->depth = depth;
  S->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) {
    // freed request memory stays in the pool for the next request
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, S->device);
    if (e == cudaSuccess) {
      uint64_t keep = static_cast<uint64_t>(hbm_budget_bytes);
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(nullptr, e, "cb_server_create");
  }
  S->admitter = std::thread(admitter_loop, S);
  S->stepper = std::thread(stepper_loop, S);
  *out = S;
  return CB_OK;
}

int cb_server_submit(cb_server_t s, int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                     uint32_t supersteps, int64_t* id) {
  if (!s || !id || n < 0 || n > 0x7fffffffLL || !row_ptr) return fail(nullptr, CB_EINVAL, "cb_server_submit: bad argument");
  const int64_t nnz = row_ptr[n];
  if (row_ptr[0] != 0 || nnz < 0 || (nnz > 0 && !col)) return fail(nullptr, CB_EINVAL, "cb_server_submit: bad row_ptr");
  auto r = std::make_shared<Request>();
  r->n = n;
  r->nnz = nnz;
  r->seed = seed;
  r->steps = supersteps;
  r->rp.assign(row_ptr, row_ptr + n + 1);
  r->col.assign(col, col + nnz);
  for (int64_t x = 0; x < n; ++x) r->maxdeg = std::max(r->maxdeg, row_ptr[x + 1] - row_ptr[x]);
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, s->device);
  r->est = estimate_handle_bytes(n, nnz, r->maxdeg, dev_sms);
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t[0] = s->now();
  s->all[r->id] = r;
  s->queue.push_back(r);
  ++s->n_submitted;
  s->cv_admit.notify_all();
  *id = r->id;
  return CB_OK;
}

int cb_server_poll(cb_server_t s, int64_t* ids, int32_t capacity, int32_t timeout_ms) {
  if (!s || (capacity > 0 && !ids) || capacity < 0) return fail(nullptr, CB_EINVAL, "cb_server_poll: bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done_ids.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done_ids.empty(); });
  int k = 0;
  while (k < capacity && !s->done_ids.empty()) {
    ids[k++] = s->done_ids.front();
    s->done_ids.pop_front();
  }
  return k;
}

int cb_server_result(cb_server_t s, int64_t id, int32_t* edges, int64_t capacity_pairs, int64_t* m_out,
                     double* times) {
  if (!s || !m_out) return fail(nullptr, CB_EINVAL, "cb_server_result: bad argument");
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(nullptr, CB_EINVAL, "cb_server_result: unknown request id");
    r = it->second;
    if (r->st != St::Done) return fail(nullptr, CB_EINVAL, "cb_server_result: request not finished");
  }
  if (times)
    for (int i = 0; i < 4; ++i) times[i] = r->t[i];
  *m_out = r->m;
  if (r->rc != CB_OK) {
    fail(nullptr, r->rc, r->err);
    if (edges) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->all.erase(id);
    }
    return r->rc;
  }
  if (!edges) return CB_OK;
  if (capacity_pairs < r->m) return fail(nullptr, CB_ESIZE, "cb_server_result: capacity below m");
  if (r->m) std::memcpy(edges, r->edges.data(), sizeof(int32_t) * 2 * static_cast<size_t>(r->m));
  std::lock_guard<std::mutex> lk(s->mu);
  s->all.erase(id);
  return CB_OK;
}

int cb_server_stats(cb_server_t s, int64_t* out, int32_t count) {
  if (!s || !out || count < 0) return fail(nullptr, CB_EINVAL, "cb_server_stats: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t v[8] = {s->n_submitted, static_cast<int64_t>(s->queue.size()), s->n_resident, s->n_done,
                        s->reserved, s->reserved_peak, s->steps_issued, s->n_failed};
  const int k = std::min(count, 8);
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return k;
}

void cb_server_destroy(cb_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_admit.notify_all();
    s->cv_step.notify_all();
    s->cv_done.notify_all();
  }
  if (s->admitter.joinable()) s->admitter.join();
  if (s->stepper.joinable()) s->stepper.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->all) release_request_device(kv.second.get());
  delete s;
}

}  // extern "C"
