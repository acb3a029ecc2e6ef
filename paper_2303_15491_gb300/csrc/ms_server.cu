// Serving: a request loop that admits segmentations of mixed sizes as slots
// and device memory free up, and runs them concurrently on the GPU.
//
// Each slot is a host worker thread with its own ms_ctx (own stream and own
// resident scratch), so the kernels of different requests overlap on the
// device.  The budget covers everything the server's requests hold on the
// device: the scratch every slot keeps between requests (measured after each
// request), and for each running request its field and labels plus the
// scratch growth it is estimated to cause in its slot.  A request is admitted
// when a slot is idle and that much fits in what the budget has left; among
// waiting requests the first that fits is admitted (a request that has been
// passed over kMaxBypass times blocks later ones until it fits, so large
// requests are not starved).  Idle slots give their scratch back while a
// waiting request does not fit.  Requests of at least kLargeVertices vertices
// run one at a time.
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
  size_t io_bytes;       // the caller's field and labels
  size_t scratch_bytes;  // estimated scratch of its segmentation
  size_t charged = 0;    // what admission added to in_use for it (io + growth)
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

// Device memory of one request: the caller's field and three label arrays,
// and the library's scratch (tile pair numbers, face roots, pair pool, root
// lists, pair set, sort buffers), estimated at 10 bytes per vertex.
size_t io_bytes_of(const int64_t dims[3], ms_dtype dtype) {
  const size_t n = (size_t)(dims[0] * dims[1] * dims[2]);
  return n * ((dtype == MS_F16 ? 2 : 4) + 12);
}
size_t scratch_estimate(const int64_t dims[3]) {
  const size_t n = (size_t)(dims[0] * dims[1] * dims[2]);
  return n * 10 + ((size_t)64 << 20);
}

}  // namespace

struct ms_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;  // slots' resident scratch + running requests' charges
  size_t peak = 0;
  std::vector<size_t> resident;  // per slot: device bytes its context holds
  std::vector<char> busy;        // per slot: running a request
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

size_t growth_of(const Request &r, size_t resident) {
  return r.scratch_bytes > resident ? r.scratch_bytes - resident : 0;
}

// Pop the first request admissible on idle slot `slot` (caller holds mu);
// false if none fits.
bool take_admissible(ms_server *s, int slot, Request *out) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->large && s->large_running > 0) continue;  // waits for the running large one
    const size_t need = it->io_bytes + growth_of(*it, s->resident[slot]);
    if (s->in_use + need <= s->budget) {
      *out = *it;
      out->charged = need;
      // everything ahead of it was passed over once more
      for (auto jt = s->queue.begin(); jt != it; ++jt) jt->bypassed++;
      s->queue.erase(it);
      s->in_use += need;
      s->large_running += out->large ? 1 : 0;
      if (s->in_use > s->peak) s->peak = s->in_use;
      s->admitted++;
      return true;
    }
    if (it->bypassed >= kMaxBypass) return false;  // it goes first once it fits
  }
  return false;
}

void worker_main(ms_server *s, int slot) {
  cudaSetDevice(s->device);
  ms_ctx *ctx = s->ctxs[slot];
  for (;;) {
    Request r{};
    bool release = false;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] {
        if (s->stopping || take_admissible(s, slot, &r)) return true;
        // a waiting request does not fit and nothing runs that could free
        // memory: an idle slot gives its scratch back
        if (!s->queue.empty() && s->resident[slot] > sizeof(msseg::DevStatus)) {
          bool any_busy = false;
          for (char b : s->busy) any_busy = any_busy || b;
          if (!any_busy) {
            release = true;
            return true;
          }
        }
        return false;
      });
      if (s->stopping && r.ticket == 0) return;
      s->busy[slot] = 1;  // running a request, or its context is being freed
    }
    if (release) {
      msseg::ctx_release_scratch(ctx);
      const size_t now_resident = msseg::ctx_resident_bytes(ctx);
      {
        std::lock_guard<std::mutex> lock(s->mu);
        s->in_use = s->in_use - s->resident[slot] + now_resident;
        s->resident[slot] = now_resident;
        s->busy[slot] = 0;
      }
      s->cv_work.notify_all();
      s->cv_done.notify_all();
      continue;
    }
    int64_t k = 0;
    const long long l0 = msseg::tl_launches;  // this worker thread's launch counter
    ms_status st = ms_segment(ctx, r.field, r.dims, r.dtype, r.asc, r.desc, r.ms);
    const long long nl = msseg::tl_launches - l0;
    if (st == MS_OK) ms_last_region_count(ctx, &k);
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r.submitted).count();
    size_t now_resident = msseg::ctx_resident_bytes(ctx);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      // the estimate becomes the measured size of the slot's scratch
      s->in_use -= r.charged;
      s->in_use = s->in_use - s->resident[slot] + now_resident;
      s->resident[slot] = now_resident;
      if (s->in_use > s->peak) s->peak = s->in_use;
      release = s->in_use > s->budget;  // grew beyond its estimate
    }
    if (release) {
      msseg::ctx_release_scratch(ctx);
      now_resident = msseg::ctx_resident_bytes(ctx);
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (release) {
        s->in_use = s->in_use - s->resident[slot] + now_resident;
        s->resident[slot] = now_resident;
      }
      Result &res = s->results[r.ticket];
      res.done = true;
      res.status = st;
      res.k = k;
      res.latency_ms = ms;
      s->large_running -= r.large ? 1 : 0;
      s->busy[slot] = 0;
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
  s->resident.assign(s->ctxs.size(), 0);
  s->busy.assign(s->ctxs.size(), 0);
  for (size_t i = 0; i < s->ctxs.size(); ++i) {
    s->resident[i] = msseg::ctx_resident_bytes(s->ctxs[i]);
    s->in_use += s->resident[i];
  }
  s->peak = s->in_use;
  for (size_t i = 0; i < s->ctxs.size(); ++i) s->workers.emplace_back(worker_main, s, (int)i);
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
  r.io_bytes = io_bytes_of(dims, dtype);
  r.scratch_bytes = scratch_estimate(dims);
  r.large = dims[0] * dims[1] * dims[2] >= kLargeVertices;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return MS_ERR_INVALID_ARG;
    // could never be admitted, even with every slot's scratch given back
    if (r.io_bytes + r.scratch_bytes + sizeof(msseg::DevStatus) * s->ctxs.size() > s->budget)
      return MS_ERR_TOO_LARGE;
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
  // a ticket another waiter has already released counts as ready (and is
  // then reported as unknown)
  auto ready = [&] {
    auto jt = s->results.find(ticket);
    return jt == s->results.end() || jt->second.done;
  };
  if (timeout_ms < 0)
    s->cv_done.wait(lock, ready);
  else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready))
    return MS_ERR_TIMEOUT;
  it = s->results.find(ticket);
  if (it == s->results.end()) return MS_ERR_INVALID_ARG;
  Result r = it->second;
  s->results.erase(it);
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
  size_t res = 0;
  for (size_t x : s->resident) res += x;
  out->resident_bytes = res;
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
    s->cv_done.wait(lock, [&] {
      if (!s->queue.empty()) return false;
      for (char b : s->busy)
        if (b) return false;
      return true;
    });
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (std::thread &t : s->workers) t.join();
  for (ms_ctx *c : s->ctxs) ms_destroy(c);
  delete s;
  return MS_OK;
}

}  // extern "C"
