// Serving: a request loop that admits segmentations of mixed sizes as slots
// and device memory free up, and runs them concurrently on the GPU.
//
// Each slot is a host worker thread with its own ms_ctx (own stream and own
// resident scratch), so the kernels of different requests overlap on the
// device.  A request is admitted when a slot is idle and its estimated device
// memory (its field and labels plus the scratch its segmentation needs) fits
// in what the budget has left; among waiting requests the first that fits is
// admitted (a request that has been passed over kMaxBypass times blocks
// later ones until it fits, so large requests are not starved).  Requests of
// at least kLargeVertices vertices run one at a time.
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ms_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxBypass = 8;
// A request this large fills the GPU by itself: two of them side by side only
// slow each other down, so at most one runs at a time (smaller requests still
// run beside it).
constexpr int64_t kLargeVertices = 1ll << 25;

struct Request {
  uint64_t ticket = 0;
  const void *field;
  int64_t dims[3];
  ms_dtype dtype;
  int32_t *asc, *desc, *ms;
  size_t bytes;  // admission estimate
  bool large = false;
  int bypassed = 0;
  Clock::time_point submitted;
};

struct Result {
  bool done = false;
  ms_status status = MS_OK;
  int64_t k = 0;
  double latency_ms = 0.0;
};

// Estimated device memory of one request: the caller's field and three label
// arrays, and the library's scratch (tile pair numbers, face roots, pair pool,
// pair set, sort buffers), about 10 bytes per vertex.
size_t estimate_bytes(const int64_t dims[3], ms_dtype dtype) {
  const size_t n = (size_t)(dims[0] * dims[1] * dims[2]);
  const size_t esz = dtype == MS_F16 ? 2 : 4;
  return n * (esz + 12 + 10) + ((size_t)64 << 20);
}

}  // namespace

struct ms_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  size_t peak = 0;
  int large_running = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
  uint64_t admitted = 0, completed = 0;
  uint64_t launches = 0;  // kernel launches of completed requests
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Result> results;
  std::vector<std::thread> workers;
  std::vector<ms_ctx *> ctxs;
};

namespace {

// Pop the first admissible request (caller holds mu); false if none fits.
bool take_admissible(ms_server *s, Request *out) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->large && s->large_running > 0) continue;  // waits for the running large one
    if (s->in_use + it->bytes <= s->budget) {
      *out = *it;
      // everything ahead of it was passed over once more
      for (auto jt = s->queue.begin(); jt != it; ++jt) jt->bypassed++;
      s->queue.erase(it);
      s->in_use += out->bytes;
      s->large_running += out->large ? 1 : 0;
      if (s->in_use > s->peak) s->peak = s->in_use;
      s->admitted++;
      return true;
    }
    if (it->bypassed >= kMaxBypass) return false;  // it goes first once it fits
  }
  return false;
}

void worker_main(ms_server *s, ms_ctx *ctx) {
  cudaSetDevice(s->device);
  for (;;) {
    Request r{};
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stopping || take_admissible(s, &r); });
      if (s->stopping && r.ticket == 0) return;
    }
    int64_t k = 0;
    const long long l0 = msseg::tl_launches;  // this worker thread's launch counter
    ms_status st = ms_segment(ctx, r.field, r.dims, r.dtype, r.asc, r.desc, r.ms);
    const long long nl = msseg::tl_launches - l0;
    if (st == MS_OK) ms_last_region_count(ctx, &k);
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r.submitted).count();
    {
      std::lock_guard<std::mutex> lock(s->mu);
      Result &res = s->results[r.ticket];
      res.done = true;
      res.status = st;
      res.k = k;
      res.latency_ms = ms;
      s->in_use -= r.bytes;
      s->large_running -= r.large ? 1 : 0;
      s->completed++;
      s->launches += (uint64_t)nl;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // freed budget may admit waiting requests
  }
}

}  // namespace

extern "C" {

ms_status ms_server_create(ms_server **out, int device, size_t budget_bytes, int n_slots) {
  if (!out || n_slots < 1 || n_slots > 64 || budget_bytes == 0) return MS_ERR_INVALID_ARG;
  ms_server *s = new (std::nothrow) ms_server();
  if (!s) return MS_ERR_OUT_OF_MEMORY;
  s->device = device;
  s->budget = budget_bytes;
  for (int i = 0; i < n_slots; ++i) {
    ms_ctx *c = nullptr;
    const ms_status st = ms_create(&c, device, nullptr);
    if (st != MS_OK) {
      for (ms_ctx *x : s->ctxs) ms_destroy(x);
      delete s;
      return st;
    }
    s->ctxs.push_back(c);
  }
  for (ms_ctx *c : s->ctxs) s->workers.emplace_back(worker_main, s, c);
  *out = s;
  return MS_OK;
}

ms_status ms_server_submit(ms_server *s, const void *field, const int64_t dims[3], ms_dtype dtype,
                           int32_t *out_asc, int32_t *out_desc, int32_t *out_ms, uint64_t *ticket) {
  if (!s || !field || !dims || !out_asc || !out_desc || !out_ms || !ticket)
    return MS_ERR_INVALID_ARG;
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return MS_ERR_INVALID_ARG;
  if (dtype != MS_F32 && dtype != MS_F16) return MS_ERR_UNSUPPORTED_DTYPE;
  Request r;
  r.field = field;
  for (int i = 0; i < 3; ++i) r.dims[i] = dims[i];
  r.dtype = dtype;
  r.asc = out_asc;
  r.desc = out_desc;
  r.ms = out_ms;
  r.bytes = estimate_bytes(dims, dtype);
  r.large = dims[0] * dims[1] * dims[2] >= kLargeVertices;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return MS_ERR_INVALID_ARG;
    if (r.bytes > s->budget) return MS_ERR_TOO_LARGE;  // could never be admitted
    r.ticket = s->next_ticket++;
    s->results[r.ticket] = Result{};
    s->queue.push_back(r);
    *ticket = r.ticket;
  }
  s->cv_work.notify_all();
  return MS_OK;
}

ms_status ms_server_wait(ms_server *s, uint64_t ticket, int64_t timeout_ms, ms_status *result,
                         int64_t *k_out, double *latency_ms) {
  if (!s) return MS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return MS_ERR_INVALID_ARG;
  auto ready = [&] { return s->results[ticket].done; };
  if (timeout_ms < 0)
    s->cv_done.wait(lock, ready);
  else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready))
    return MS_ERR_TIMEOUT;
  Result r = s->results[ticket];
  s->results.erase(ticket);
  if (result) *result = r.status;
  if (k_out) *k_out = r.k;
  if (latency_ms) *latency_ms = r.latency_ms;
  return MS_OK;
}

ms_status ms_server_stats(ms_server *s, ms_server_info *out) {
  if (!s || !out) return MS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->queued = s->queue.size();
  out->bytes_in_use = s->in_use;
  out->peak_bytes = s->peak;
  out->budget_bytes = s->budget;
  out->launches = s->launches;
  return MS_OK;
}

ms_status ms_server_destroy(ms_server *s) {
  if (!s) return MS_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    // finish everything already submitted
    s->cv_done.wait(lock, [&] { return s->queue.empty() && s->in_use == 0; });
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (std::thread &t : s->workers) t.join();
  for (ms_ctx *c : s->ctxs) ms_destroy(c);
  delete s;
  return MS_OK;
}

}  // extern "C"
