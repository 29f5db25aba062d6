// Served form: a request loop with continuous batching over resident sets.
//
// Callers submit point-batch requests (host buffers) for any resident set.
// A dispatcher thread owns n_streams slots; each slot has a stream, device
// staging buffers, pinned staging buffers and a batched plan (one persistent
// graph launch for all requests of a launch). Whenever a slot is free, the
// dispatcher admits queued requests into it while the slot's point and
// request capacity allow (the capacities come from the device-memory
// budget), copies their points in (small requests gathered on the CPU into
// pinned memory and sent in one copy, large ones copied directly), runs the
// plan and copies the ids back. Requests that arrive while launches are in
// flight wait only for the next free slot, so their work overlaps the
// running launches (continuous batching). Each launch ends with an event on
// its slot's stream; the dispatcher polls the events of busy slots (it
// spins, yielding, while launches are in flight and for a short window
// after the last activity, then sleeps until a submit wakes it), marks the
// requests done and records their latency, so a small request's completion
// takes no host callback and no extra thread hand-off. A request larger than
// one launch holds is queued as consecutive parts of at most a launch each
// (its point vector cut into ranges, Appendix A takes vectors of any
// length); its ticket completes, and its latency is recorded, when the last
// part is done.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pip_internal.cuh"

namespace pip {
pip_status plan_prepare(pip_plan plan, int64_t superbins, bool compact, cudaStream_t s);
}

namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t GATHER_MAX = 1 << 15;  // requests up to this size are gathered on the CPU
constexpr int64_t LAT_WINDOW = 1 << 22;  // latency samples kept for the percentiles
constexpr double SPIN_IDLE_US = 200.0;   // the dispatcher keeps polling this long after activity
constexpr double SPIN_WAIT_US = 300.0;   // pip_server_wait polls this long before it sleeps

struct Req {
  uint64_t ticket = 0;
  int32_t set = 0;
  const double* lon = nullptr;
  const double* lat = nullptr;
  int64_t n = 0;
  int32_t* out = nullptr;
  Clock::time_point t_sub, t_done;
  std::atomic<int> state{0};  // 0 queued, 1 running, 2 done (written under the server's lock)
  pip_status err = PIP_OK;
  int64_t off = 0;       // offset in the slot's staging buffers
  bool gathered = false;
  Req* parent = nullptr;                  // a part of a split request: the whole request
  int64_t parts_left = 0;                 // whole split request: parts not done yet
  std::vector<std::unique_ptr<Req>> parts;
};

// Mark r done (lock held); returns the request whose latency completes now,
// or nullptr while parts of a split request are still outstanding.
Req* finish_req(Req* r, Clock::time_point now, pip_status err) {
  r->t_done = now;
  r->state = 2;
  if (err != PIP_OK) r->err = err;
  Req* p = r->parent;
  if (!p) return r;
  if (err != PIP_OK) p->err = err;
  if (--p->parts_left > 0) return nullptr;
  p->t_done = now;
  p->state = 2;
  return p;
}

struct Slot;

}  // namespace

struct pip_server_s {
  int device = 0;
  std::vector<pip_set> sets;
  pip_server_opts opts{};
  int64_t cap_points = 0;
  int32_t cap_queries = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::unique_ptr<Slot>> slots;
  std::thread dispatcher;
  // stats
  std::vector<double> lat_us;  // latencies of the most recent LAT_WINDOW completions (a ring)
  int64_t lat_seen = 0;        // completions recorded since the last reset
  int64_t submitted = 0, completed = 0, rejected = 0, launches = 0, points = 0, batch_queries = 0;
};

namespace {

struct Slot {
  pip_server_s* srv = nullptr;
  cudaStream_t s = nullptr;
  pip_plan plan = nullptr;
  pip::Alloc alloc;
  pip::DBuf<double> dlon, dlat;
  pip::DBuf<int32_t> dout;
  double* hlon = nullptr;
  double* hlat = nullptr;
  int32_t* hout = nullptr;
  std::vector<Req*> batch;
  bool busy = false;
  cudaEvent_t done_ev = nullptr;  // recorded after the launch's copies back
  ~Slot() {
    if (done_ev) cudaEventDestroy(done_ev);
    if (plan) pip_plan_destroy(plan);
    if (hlon) cudaFreeHost(hlon);
    if (hlat) cudaFreeHost(hlat);
    if (hout) cudaFreeHost(hout);
    dlon.release();
    dlat.release();
    dout.release();
    if (s) cudaStreamDestroy(s);
  }
};

// The slot's launch and copies are complete (server lock held): hand the
// gathered ids back, mark the requests done and record their latency.
void complete_slot(pip_server_s* S, Slot* sl, pip_status err) {
  const auto now = Clock::now();
  for (Req* part : sl->batch) {
    if (err == PIP_OK && part->gathered && part->n > 0)
      std::memcpy(part->out, sl->hout + part->off, part->n * sizeof(int32_t));
    Req* r = finish_req(part, now, err);
    if (!r || r->err != PIP_OK) continue;  // a failed request (any of its parts) is not a completion
    const double us = std::chrono::duration<double, std::micro>(r->t_done - r->t_sub).count();
    if ((int64_t)S->lat_us.size() < LAT_WINDOW) S->lat_us.push_back(us);
    else S->lat_us[S->lat_seen % LAT_WINDOW] = us;
    ++S->lat_seen;
    ++S->completed;
  }
  sl->batch.clear();
  sl->busy = false;
  S->cv.notify_all();
}

// Stage, run and copy back one admitted batch on a slot (no lock held).
pip_status launch_batch(pip_server_s* S, Slot* sl) {
  cudaStream_t s = sl->s;
  std::vector<pip_query> qs;
  qs.reserve(sl->batch.size());
  int64_t off = 0, g_lo = -1, g_hi = 0;
  for (Req* r : sl->batch) {
    r->off = off;
    r->gathered = r->n <= GATHER_MAX;
    if (r->n > 0) {
      if (r->gathered) {
        std::memcpy(sl->hlon + off, r->lon, r->n * sizeof(double));
        std::memcpy(sl->hlat + off, r->lat, r->n * sizeof(double));
        if (g_lo < 0) g_lo = off;
        g_hi = off + r->n;
      }
    }
    qs.push_back(pip_query{S->sets[r->set], sl->dlon.p + off, sl->dlat.p + off, r->n, sl->dout.p + off});
    off += r->n;
  }
  // gathered requests: one copy of the pinned range (it may also cover direct
  // requests' slots, which their own copies overwrite afterwards)
  if (g_lo >= 0) {
    PIP_CUDA(cudaMemcpyAsync(sl->dlon.p + g_lo, sl->hlon + g_lo, (g_hi - g_lo) * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    PIP_CUDA(cudaMemcpyAsync(sl->dlat.p + g_lo, sl->hlat + g_lo, (g_hi - g_lo) * sizeof(double),
                             cudaMemcpyHostToDevice, s));
  }
  for (Req* r : sl->batch) {
    if (r->gathered || r->n == 0) continue;
    PIP_CUDA(cudaMemcpyAsync(sl->dlon.p + r->off, r->lon, r->n * sizeof(double), cudaMemcpyDefault, s));
    PIP_CUDA(cudaMemcpyAsync(sl->dlat.p + r->off, r->lat, r->n * sizeof(double), cudaMemcpyDefault, s));
  }
  pip_status st = pip_plan_run(sl->plan, qs.data(), (int32_t)qs.size(), s);
  if (st != PIP_OK) return st;
  if (g_lo >= 0)
    PIP_CUDA(cudaMemcpyAsync(sl->hout + g_lo, sl->dout.p + g_lo, (g_hi - g_lo) * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s));
  for (Req* r : sl->batch) {
    if (r->gathered || r->n == 0) continue;
    PIP_CUDA(cudaMemcpyAsync(r->out, sl->dout.p + r->off, r->n * sizeof(int32_t), cudaMemcpyDefault, s));
  }
  PIP_CUDA(cudaEventRecord(sl->done_ev, s));
  return PIP_OK;
}

void dispatch_loop(pip_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  auto active = Clock::now();
  while (true) {
    // completions of busy slots
    bool any_busy = false;
    for (auto& sl : S->slots) {
      if (!sl->busy) continue;
      const cudaError_t q = cudaEventQuery(sl->done_ev);
      if (q == cudaSuccess) {
        complete_slot(S, sl.get(), PIP_OK);
        active = Clock::now();
      } else if (q == cudaErrorNotReady) {
        cudaGetLastError();  // not an error: clear it from this thread's state
        any_busy = true;
      } else {
        cudaGetLastError();
        complete_slot(S, sl.get(), PIP_ECUDA);
      }
    }
    if (S->stop && S->pending.empty() && !any_busy) break;
    Slot* free_slot = nullptr;
    for (auto& sl : S->slots)
      if (!sl->busy) {
        free_slot = sl.get();
        break;
      }
    if (S->pending.empty() || !free_slot) {
      const double idle_us = std::chrono::duration<double, std::micro>(Clock::now() - active).count();
      if (any_busy || idle_us < SPIN_IDLE_US) {  // keep polling, without holding the lock
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      } else {
        S->cv.wait(lk);
        active = Clock::now();
      }
      continue;
    }
    // admit queued requests while the slot's capacities allow
    int64_t pts = 0;
    while (!S->pending.empty() && (int32_t)free_slot->batch.size() < S->cap_queries) {
      Req* r = S->pending.front();
      if (pts + r->n > S->cap_points && !free_slot->batch.empty()) break;
      S->pending.pop_front();
      r->state = 1;
      free_slot->batch.push_back(r);
      pts += r->n;
    }
    free_slot->busy = true;
    ++S->launches;
    S->points += pts;
    S->batch_queries += (int64_t)free_slot->batch.size();
    lk.unlock();
    pip_status st = launch_batch(S, free_slot);
    lk.lock();
    active = Clock::now();
    if (st != PIP_OK) {  // fail the batch's requests; the slot stays usable
      cudaStreamSynchronize(free_slot->s);  // nothing of the failed launch stays in flight
      cudaGetLastError();
      complete_slot(S, free_slot, st);
    }
  }
}

}  // namespace

using namespace pip;

extern "C" pip_status pip_server_create(const pip_set* sets, int32_t n_sets, const pip_server_opts* opts,
                                        pip_server* out) {
  if (!out) return fail(PIP_EINVAL, "pip_server_create: out is NULL");
  *out = nullptr;
  if (!sets || n_sets <= 0 || n_sets > 64) return fail(PIP_EINVAL, "pip_server_create: 1..64 sets");
  for (int i = 0; i < n_sets; ++i)
    if (!sets[i]) return fail(PIP_EINVAL, "pip_server_create: NULL set");
  std::unique_ptr<pip_server_s> S(new pip_server_s());
  PIP_CUDA(cudaGetDevice(&S->device));
  S->sets.assign(sets, sets + n_sets);
  if (opts) S->opts = *opts;
  pip_server_opts& o = S->opts;
  if (o.n_streams <= 0) o.n_streams = 2;
  if (o.max_batch_queries <= 0) o.max_batch_queries = 1024;
  if (o.max_batch_points <= 0) o.max_batch_points = 1 << 24;
  if (o.max_pending <= 0) o.max_pending = 1 << 20;
  // device bytes per point of one slot: staging (8 + 8 + 4) + plan (2 x 16)
  const int64_t per_point = 52;
  if (o.mem_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    PIP_CUDA(cudaMemGetInfo(&fr, &tot));
    o.mem_budget_bytes = (int64_t)(fr / 4);
  }
  S->cap_points = std::min<int64_t>(o.max_batch_points, o.mem_budget_bytes / (per_point * o.n_streams));
  if (S->cap_points < 1) return fail(PIP_ENOMEM, "pip_server_create: memory budget too small");
  S->cap_queries = o.max_batch_queries;
  int64_t superbins = 0;
  bool compact = false;
  for (pip_set set : S->sets) {
    superbins += std::max<int64_t>(1, set->view.n_sb);
    compact |= set->view.compact != 0;
  }
  for (int i = 0; i < o.n_streams; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->srv = S.get();
    PIP_CUDA(cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking));
    PIP_CUDA(cudaEventCreateWithFlags(&sl->done_ev, cudaEventDisableTiming));
    pip_status st = pip_plan_create(S->cap_points, S->cap_queries, sl->s, &sl->plan);
    if (st != PIP_OK) return st;
    // buffers for every resident set at once and both graphs captured now:
    // no batch allocates or captures mid-service
    st = plan_prepare(sl->plan, superbins, compact, sl->s);
    if (st != PIP_OK) return st;
    if (!sl->dlon.alloc(&sl->alloc, S->cap_points, sl->s) || !sl->dlat.alloc(&sl->alloc, S->cap_points, sl->s) ||
        !sl->dout.alloc(&sl->alloc, S->cap_points, sl->s))
      return fail(PIP_ENOMEM, "pip_server_create: staging");
    PIP_CUDA(cudaMallocHost((void**)&sl->hlon, S->cap_points * sizeof(double)));
    PIP_CUDA(cudaMallocHost((void**)&sl->hlat, S->cap_points * sizeof(double)));
    PIP_CUDA(cudaMallocHost((void**)&sl->hout, S->cap_points * sizeof(int32_t)));
    PIP_CUDA(cudaStreamSynchronize(sl->s));
    S->slots.push_back(std::move(sl));
  }
  S->dispatcher = std::thread(dispatch_loop, S.get());
  *out = S.release();
  return PIP_OK;
}

extern "C" pip_status pip_server_submit(pip_server srv, int32_t set, const double* lon, const double* lat,
                                        int64_t n, int32_t* out, uint64_t* ticket) {
  if (!srv || !ticket) return fail(PIP_EINVAL, "pip_server_submit: NULL argument");
  if (set < 0 || set >= (int32_t)srv->sets.size()) return fail(PIP_EINVAL, "pip_server_submit: bad set");
  if (n < 0 || (n > 0 && (!lon || !lat || !out))) return fail(PIP_EINVAL, "pip_server_submit: bad buffers");
  const int64_t cap = srv->cap_points;
  const int64_t n_parts = n > cap ? (n + cap - 1) / cap : 1;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return fail(PIP_EINVAL, "pip_server_submit: server is stopping");
  if ((int64_t)srv->pending.size() + n_parts > srv->opts.max_pending) {
    ++srv->rejected;
    return fail(PIP_EBUSY, "pip_server_submit: queue full");
  }
  auto r = std::make_unique<Req>();
  r->ticket = srv->next_ticket++;
  r->set = set;
  r->lon = lon;
  r->lat = lat;
  r->n = n;
  r->out = out;
  r->t_sub = Clock::now();
  *ticket = r->ticket;
  if (n_parts == 1) {
    srv->pending.push_back(r.get());
  } else {  // consecutive ranges of at most one launch each
    r->parts_left = n_parts;
    for (int64_t k = 0; k < n_parts; ++k) {
      auto q = std::make_unique<Req>();
      const int64_t a = k * cap, m = std::min(cap, n - a);
      q->ticket = r->ticket;
      q->set = set;
      q->lon = lon + a;
      q->lat = lat + a;
      q->n = m;
      q->out = out + a;
      q->t_sub = r->t_sub;
      q->parent = r.get();
      srv->pending.push_back(q.get());
      r->parts.push_back(std::move(q));
    }
  }
  srv->reqs.emplace(r->ticket, std::move(r));
  ++srv->submitted;
  srv->cv.notify_all();
  return PIP_OK;
}

extern "C" pip_status pip_server_wait(pip_server srv, uint64_t ticket, int64_t timeout_us) {
  if (!srv) return fail(PIP_EINVAL, "pip_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(PIP_EINVAL, "pip_server_wait: unknown ticket");
  Req* r = it->second.get();
  auto done = [&] { return r->state == 2; };
  if (!done()) {  // poll a little before sleeping: small requests finish within it
    lk.unlock();
    const auto t0 = Clock::now();
    const double limit = timeout_us < 0 ? SPIN_WAIT_US : std::min<double>(SPIN_WAIT_US, (double)timeout_us);
    while (r->state.load(std::memory_order_acquire) != 2 &&
           std::chrono::duration<double, std::micro>(Clock::now() - t0).count() < limit)
      std::this_thread::yield();
    lk.lock();
  }
  if (timeout_us < 0) {
    srv->cv.wait(lk, done);
  } else if (!srv->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    return fail(PIP_ETIMEOUT, "pip_server_wait: not done yet");
  }
  const pip_status st = r->err;
  srv->reqs.erase(it);
  if (st != PIP_OK) return fail(st, "pip_server_wait: the request's launch failed");
  return PIP_OK;
}

extern "C" pip_status pip_server_stats(pip_server srv, pip_server_stats_t* st, int32_t reset) {
  if (!srv || !st) return fail(PIP_EINVAL, "pip_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  st->submitted = srv->submitted;
  st->completed = srv->completed;
  st->rejected = srv->rejected;
  st->launches = srv->launches;
  st->points = srv->points;
  st->mean_batch_queries = srv->launches ? (double)srv->batch_queries / srv->launches : 0.0;
  std::vector<double> v = srv->lat_us;
  if (!v.empty()) {
    auto pct = [&](double p) {
      const size_t k = std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return v[k];
    };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    st->max_us = *std::max_element(v.begin(), v.end());
  } else {
    st->p50_us = st->p99_us = st->max_us = 0.0;
  }
  if (reset) {
    srv->lat_us.clear();
    srv->lat_seen = 0;
    srv->submitted = srv->completed = srv->rejected = srv->launches = srv->points = 0;
    srv->batch_queries = 0;
  }
  return PIP_OK;
}

extern "C" void pip_server_destroy(pip_server srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->dispatcher.joinable()) srv->dispatcher.join();
  for (auto& sl : srv->slots) cudaStreamSynchronize(sl->s);
  srv->slots.clear();
  delete srv;
}
