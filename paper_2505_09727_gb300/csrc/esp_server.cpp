// Request server: resident systems, memory-budgeted plans, continuous
// batching of force/energy requests on one device (include/esp.h).
//
// Every system is registered once (box, N, charges). A request names a
// system, a tolerance and a set of positions. A worker thread keeps up to
// max_inflight requests on the device at once: each runs on the resident plan
// of its (system, tolerance) on that plan's own streams, so requests for
// different systems overlap on the device, and a request that arrives while
// others run is started as soon as a slot, its plan and the memory for it are
// free. Plans (sorted bins, grids, FFT plans) stay resident across requests;
// when a new plan would exceed the memory budget, idle plans are destroyed in
// least-recently-used order. Inputs and outputs pass through pinned host
// buffers, so a whole request (copies and kernels) is asynchronous.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/esp.h"
#include "esp_engine.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

esp_status sfail(esp_status s, const std::string& m) {
  espe::set_last_error(m);
  return s;
}

// Pinned host buffers, reused by size class (powers of two).
class PinnedPool {
 public:
  ~PinnedPool() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
  }
  void* get(size_t bytes, size_t* cls_out) {
    size_t cls = 4096;
    while (cls < bytes) cls <<= 1;
    *cls_out = cls;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto& v = free_[cls];
      if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        return p;
      }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, cls, cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cls) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_[cls].push_back(p);
  }

 private:
  std::mutex mu_;
  std::map<size_t, std::vector<void*>> free_;
};

struct SystemRec {
  esp_box box;
  int64_t N;
  std::vector<double> q;
};

struct PlanRec {
  int sys = -1;
  double tol = 0;
  esp_plan_t plan = nullptr;
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
  int64_t ticket = 0;
  int sys = 0;
  double tol = 0;
  int64_t N = 0;
  double* buf = nullptr;     // pinned: xyz[3N] | forces[3N] | potential[N] | energy | err
  size_t cls = 0;
  cudaEvent_t ev = nullptr;      // recorded after the request's last copy
  cudaEvent_t ev_start = nullptr;  // recorded before its first copy (device interval)
  PlanRec* plan = nullptr;
  PlanRec* late_plan = nullptr;   // timed out with its work still on the device: the plan it holds
  bool released = false;     // the client has taken the (timed-out) result: free once the work is done
  ReqState state = kPending;
  esp_status status = ESP_OK;
  std::string msg;
  Clock::time_point t_submit, t_start, t_done;
  double* xyz() { return buf; }
  double* forces() { return buf + 3 * N; }
  double* potential() { return buf + 6 * N; }
  double* energy() { return buf + 7 * N; }
  int* err() { return reinterpret_cast<int*>(buf + 7 * N + 1); }
};

size_t request_bytes(int64_t N) { return (size_t)(7 * N + 2) * sizeof(double); }

}  // namespace

struct esp_server_s {
  esp_server_opts opts{};
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_done;     // a request finished
  std::condition_variable cv_work;     // new request or a slot freed
  std::atomic<uint64_t> n_submitted{0};  // read by the worker while it polls unlocked
  std::thread worker;
  bool stop = false;
  std::vector<SystemRec> systems;
  std::map<std::pair<int, double>, std::unique_ptr<PlanRec>> plans;
  size_t used = 0;
  uint64_t use_clock = 0;
  std::deque<Request*> pending;
  std::vector<Request*> running;
  std::vector<Request*> late;          // timed out, work still in flight (their plans stay busy)
  std::unordered_map<int64_t, std::unique_ptr<Request>> tickets;
  int64_t next_ticket = 1;
  PinnedPool pinned;
  // statistics
  int64_t completed = 0, failed = 0, plans_created = 0, evictions = 0;
  double atoms_done = 0;
  std::vector<double> latencies;       // ms, completed requests in completion order
  cudaEvent_t ev_ref = nullptr;        // time origin of the device intervals
  std::vector<std::pair<double, double>> intervals;   // device [start, done] ms of completed requests
  int64_t peak_inflight = 0;
  Clock::time_point t_first_submit{}, t_last_done{};
  bool any_submit = false;
};

namespace {

// Destroy idle plans (least recently used first) until `need` more bytes fit.
bool make_room(esp_server_s* s, size_t need) {
  while (s->used + need > s->budget) {
    PlanRec* victim = nullptr;
    std::pair<int, double> key;
    for (auto& kv : s->plans) {
      PlanRec* pr = kv.second.get();
      if (pr->busy) continue;
      if (!victim || pr->last_use < victim->last_use) {
        victim = pr;
        key = kv.first;
      }
    }
    if (!victim) return false;
    esp_destroy(victim->plan);
    s->used -= std::min(s->used, victim->bytes);
    s->plans.erase(key);
    ++s->evictions;
  }
  return true;
}

// Plan of (system, tolerance), created if absent. Called with s->mu held.
// Returns ESP_OK with *out, ESP_ERR_BUSY when it cannot fit right now
// (*never set when it cannot fit the budget at all).
esp_status acquire_plan(esp_server_s* s, int sys, double tol, PlanRec** out, bool* never) {
  *never = false;
  const auto key = std::make_pair(sys, tol);
  auto it = s->plans.find(key);
  if (it != s->plans.end()) {
    *out = it->second.get();
    return ESP_OK;
  }
  const SystemRec& S = s->systems[sys];
  esp_plan_opts o;
  esp_plan_opts_init(&o);
  o.r_c = s->opts.r_c;
  o.precision = s->opts.precision;
  o.kernel = s->opts.kernel;
  o.device = s->opts.device;
  // the plan's own synchronous waits (creation, charges) keep the default
  // deadline; the server's deadline applies to each request's device work
  o.timeout_ms = std::max(60000.0, s->opts.timeout_ms);
  esp_plan_params est;
  esp_status st = esp_plan_query(&S.box, S.N, tol, &o, &est);
  if (st != ESP_OK) return st;
  // the query's estimate excludes the FFT work areas (about the spectrum's
  // size): keep a margin
  const size_t need = est.device_bytes + est.device_bytes / 4 + (1u << 20);
  if (need > s->budget) {
    *never = true;
    return sfail(ESP_ERR_BUSY, "system does not fit the server's memory budget");
  }
  if (!make_room(s, need)) return ESP_ERR_BUSY;
  auto pr = std::make_unique<PlanRec>();
  pr->sys = sys;
  pr->tol = tol;
  st = esp_plan(&S.box, S.N, tol, &o, &pr->plan);
  if (st != ESP_OK) return st;
  st = esp_set_charges(pr->plan, S.q.data(), ESP_HOST);
  if (st != ESP_OK) {
    esp_destroy(pr->plan);
    return st;
  }
  pr->bytes = espe::plan_device_bytes(pr->plan);
  s->used += pr->bytes;
  ++s->plans_created;
  *out = pr.get();
  s->plans[key] = std::move(pr);
  return ESP_OK;
}

void finish(esp_server_s* s, Request* r, esp_status st, const std::string& msg) {
  r->status = st;
  r->msg = msg;
  r->state = st == ESP_OK ? kDone : kFailed;
  r->t_done = Clock::now();
  if (r->plan) {
    r->plan->busy = false;
    r->plan->last_use = ++s->use_clock;
  }
  if (st == ESP_OK) {
    ++s->completed;
    s->atoms_done += (double)r->N;
    s->latencies.push_back(ms_since(r->t_submit, r->t_done));
    float a = 0.f, b = 0.f;
    if (s->ev_ref && r->ev_start && cudaEventElapsedTime(&a, s->ev_ref, r->ev_start) == cudaSuccess &&
        cudaEventElapsedTime(&b, s->ev_ref, r->ev) == cudaSuccess)
      s->intervals.emplace_back((double)a, (double)b);
    cudaGetLastError();
    s->t_last_done = r->t_done;
  } else {
    ++s->failed;
  }
}

void worker_loop(esp_server_s* s) {
  cudaSetDevice(s->opts.device);
  std::unique_lock<std::mutex> lk(s->mu);
  Clock::time_point last_progress = Clock::now();
  while (!s->stop) {
    bool progress = false;
    // completions
    for (size_t k = 0; k < s->running.size();) {
      Request* r = s->running[k];
      const cudaError_t e = cudaEventQuery(r->ev);
      if (e == cudaErrorNotReady) {
        const double age = ms_since(r->t_start, Clock::now());
        const double limit = s->opts.timeout_ms > 0 ? s->opts.timeout_ms : 60000.0;
        if (age <= limit) {
          ++k;
          continue;
        }
        // the plan stays busy while its stream still holds the work: the
        // request moves to the late list, which frees the plan (and, once
        // the client has taken the result, the buffers) when it completes
        r->late_plan = r->plan;
        r->plan = nullptr;
        finish(s, r, ESP_ERR_TIMEOUT, "request exceeded the server deadline");
        s->late.push_back(r);
      } else if (e != cudaSuccess) {
        finish(s, r, ESP_ERR_CUDA, std::string("request: ") + cudaGetErrorString(e));
      } else {
        const int flag = *r->err();
        if (flag & 1) finish(s, r, ESP_ERR_NONFINITE, "a position is NaN or infinite");
        else if (flag) finish(s, r, ESP_ERR_INTERNAL, "a kernel bounds check failed");
        else finish(s, r, ESP_OK, "");
      }
      s->running.erase(s->running.begin() + k);
      progress = true;
    }
    // late requests whose work has now left the device give their plan back
    for (size_t k = 0; k < s->late.size();) {
      Request* r = s->late[k];
      if (cudaEventQuery(r->ev) == cudaErrorNotReady) {
        ++k;
        continue;
      }
      cudaGetLastError();
      r->late_plan->busy = false;
      r->late_plan->last_use = ++s->use_clock;
      r->late_plan = nullptr;
      s->late.erase(s->late.begin() + k);
      if (r->released) {
        s->pinned.put(r->buf, r->cls);
        cudaEventDestroy(r->ev);
        if (r->ev_start) cudaEventDestroy(r->ev_start);
        s->tickets.erase(r->ticket);
      }
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admissions, oldest first; a request whose plan is busy waits its turn
    const int max_inflight = s->opts.max_inflight > 0 ? s->opts.max_inflight : 8;
    for (auto it = s->pending.begin(); it != s->pending.end() && (int)s->running.size() < max_inflight;) {
      Request* r = *it;
      PlanRec* pr = nullptr;
      bool never = false;
      esp_status st = acquire_plan(s, r->sys, r->tol, &pr, &never);
      if (st == ESP_ERR_BUSY && never) {
        finish(s, r, ESP_ERR_BUSY, "system does not fit the server's memory budget");
        it = s->pending.erase(it);
        progress = true;
        s->cv_done.notify_all();
        continue;
      }
      if (st == ESP_ERR_BUSY) {
        ++it;
        continue;
      }
      if (st != ESP_OK) {
        finish(s, r, st, esp_last_error());
        it = s->pending.erase(it);
        progress = true;
        s->cv_done.notify_all();
        continue;
      }
      if (pr->busy) {
        ++it;
        continue;
      }
      if (r->ev_start && cudaEventRecord(r->ev_start, espe::plan_stream(pr->plan)) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(r->ev_start);
        r->ev_start = nullptr;
      }
      st = espe::plan_enqueue_step(pr->plan, r->xyz(), r->forces(), r->potential(), r->energy(), r->err(), r->ev);
      if (st != ESP_OK) {
        finish(s, r, st, esp_last_error());
      } else {
        pr->busy = true;
        pr->last_use = ++s->use_clock;
        r->plan = pr;
        r->state = kRunning;
        r->t_start = Clock::now();
        s->running.push_back(r);
        s->peak_inflight = std::max<int64_t>(s->peak_inflight, (int64_t)s->running.size());
      }
      it = s->pending.erase(it);
      progress = true;
    }
    if (progress) {
      last_progress = Clock::now();
    } else {
      if (s->running.empty()) s->cv_work.wait_for(lk, std::chrono::milliseconds(s->late.empty() ? 5 : 1));
      else {
        // requests in flight: poll their completion events with the lock
        // released (clients submit and wait meanwhile), without sleeping for
        // 1 ms after the last event, then every 20 us; a new submission or
        // 200 us end the poll
        std::vector<cudaEvent_t> evs;
        evs.reserve(s->running.size());
        for (Request* r : s->running) evs.push_back(r->ev);
        const uint64_t sub0 = s->n_submitted.load(std::memory_order_acquire);
        lk.unlock();
        const Clock::time_point t0 = Clock::now();
        for (bool done = false; !done;) {
          for (cudaEvent_t e : evs)
            if (cudaEventQuery(e) != cudaErrorNotReady) done = true;
          if (done || s->n_submitted.load(std::memory_order_acquire) != sub0) break;
          const Clock::time_point now = Clock::now();
          if (now - t0 > std::chrono::microseconds(200)) break;
          if (now - last_progress < std::chrono::milliseconds(1)) std::this_thread::yield();
          else std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        lk.lock();
      }
    }
  }
}

}  // namespace

extern "C" {

void esp_server_opts_init(esp_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_inflight = 8;
  o->precision = ESP_FP32;
  o->kernel = ESP_KERNEL_PSWF;
  o->timeout_ms = 60000.0;
}

esp_status esp_server_create(const esp_server_opts* opts, esp_server_t* out) {
  if (!out) return sfail(ESP_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  esp_server_opts o;
  if (opts) o = *opts;
  else esp_server_opts_init(&o);
  if (!(o.r_c > 0)) return sfail(ESP_ERR_INVALID_ARG, "the server needs an explicit cutoff r_c");
  if (o.max_inflight < 0 || o.max_inflight > 256) return sfail(ESP_ERR_INVALID_ARG, "max_inflight must be 0 ... 256");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return sfail(ESP_ERR_CUDA, "no CUDA device available");
  }
  if (o.device < 0 || o.device >= ndev) return sfail(ESP_ERR_INVALID_ARG, "device ordinal out of range");
  esp_server_s* s = new esp_server_s();
  s->opts = o;
  size_t budget = o.memory_budget;
  if (budget == 0) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o.device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    cudaSetDevice(prev);
    budget = free_b / 10 * 8;
  }
  s->budget = budget;
  {
    // origin of the device intervals: recorded once, on the device's legacy
    // stream, before any request exists
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o.device);
    if (cudaEventCreate(&s->ev_ref) != cudaSuccess || cudaEventRecord(s->ev_ref, 0) != cudaSuccess ||
        cudaEventSynchronize(s->ev_ref) != cudaSuccess) {
      cudaGetLastError();
      if (s->ev_ref) cudaEventDestroy(s->ev_ref);
      s->ev_ref = nullptr;
    }
    cudaSetDevice(prev);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return ESP_OK;
}

esp_status esp_server_add_system(esp_server_t s, const esp_box* box, int64_t N, const double* q, int* id) {
  if (!s || !box || !q || !id) return sfail(ESP_ERR_INVALID_ARG, "NULL argument");
  if (N <= 0) return sfail(ESP_ERR_INVALID_ARG, "a system needs atoms");
  SystemRec rec;
  rec.box = *box;
  rec.N = N;
  rec.q.assign(q, q + N);
  std::lock_guard<std::mutex> lk(s->mu);
  *id = (int)s->systems.size();
  s->systems.push_back(std::move(rec));
  return ESP_OK;
}

esp_status esp_server_submit(esp_server_t s, int id, double tolerance, const double* xyz, int64_t* ticket) {
  if (!s || !xyz || !ticket) return sfail(ESP_ERR_INVALID_ARG, "NULL argument");
  int64_t N = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->systems.size()) return sfail(ESP_ERR_INVALID_ARG, "unknown system id");
    N = s->systems[id].N;
  }
  if (!(tolerance > 1e-15 && tolerance < 0.1)) return sfail(ESP_ERR_INVALID_ARG, "tolerance must be in (1e-15, 0.1)");
  auto r = std::make_unique<Request>();
  r->sys = id;
  r->tol = tolerance;
  r->N = N;
  r->buf = static_cast<double*>(s->pinned.get(request_bytes(N), &r->cls));
  if (!r->buf) return sfail(ESP_ERR_OOM, "pinned host allocation failed");
  std::memcpy(r->xyz(), xyz, (size_t)N * 3 * sizeof(double));
  {
    // timing events: their device times give the request's device interval
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->opts.device);
    const bool ok = cudaEventCreate(&r->ev) == cudaSuccess && cudaEventCreate(&r->ev_start) == cudaSuccess;
    cudaSetDevice(prev);
    if (!ok) {
      cudaGetLastError();
      if (r->ev) cudaEventDestroy(r->ev);
      s->pinned.put(r->buf, r->cls);
      return sfail(ESP_ERR_CUDA, "event creation failed");
    }
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (!s->any_submit) {
      s->any_submit = true;
      s->t_first_submit = r->t_submit;
    }
    s->pending.push_back(r.get());
    s->tickets[r->ticket] = std::move(r);
    s->n_submitted.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_one();
  return ESP_OK;
}

esp_status esp_server_poll(esp_server_t s, int64_t ticket, int* done) {
  if (!s || !done) return sfail(ESP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return sfail(ESP_ERR_INVALID_ARG, "unknown ticket");
  *done = it->second->state >= kDone;
  return ESP_OK;
}

esp_status esp_server_wait(esp_server_t s, int64_t ticket, double timeout_ms, double* energy, double* forces,
                           double* potential, double* latency_ms) {
  if (!s) return sfail(ESP_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return sfail(ESP_ERR_INVALID_ARG, "unknown ticket");
  Request* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::microseconds((long long)((timeout_ms > 0 ? timeout_ms : 60000.0) * 1000));
  while (r->state < kDone) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < kDone)
      return sfail(ESP_ERR_TIMEOUT, "request not finished before the wait deadline");
  }
  const esp_status st = r->status;
  const std::string msg = r->msg;
  if (st == ESP_OK) {
    if (energy) *energy = *r->energy();
    if (forces) std::memcpy(forces, r->forces(), (size_t)r->N * 3 * sizeof(double));
    if (potential) std::memcpy(potential, r->potential(), (size_t)r->N * sizeof(double));
    if (latency_ms) *latency_ms = ms_since(r->t_submit, r->t_done);
  }
  // a timed-out request whose copies may still land in its buffers keeps
  // them until the worker sees its work finish; the ticket is released
  if (r->late_plan) {
    r->released = true;
  } else {
    s->pinned.put(r->buf, r->cls);
    cudaEventDestroy(r->ev);
    if (r->ev_start) cudaEventDestroy(r->ev_start);
    s->tickets.erase(it);
  }
  if (st != ESP_OK) return sfail(st, msg);
  return ESP_OK;
}

esp_status esp_server_stats(esp_server_t s, esp_server_counters* out) {
  if (!s || !out) return sfail(ESP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->pending = (int64_t)s->pending.size();
  out->running = (int64_t)s->running.size();
  out->atoms_done = s->atoms_done;
  out->plans_resident = (int64_t)s->plans.size();
  out->plans_created = s->plans_created;
  out->evictions = s->evictions;
  out->device_bytes = s->used;
  out->memory_budget = s->budget;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const double x = p * (double)(v.size() - 1);
      const size_t i = (size_t)x;
      const double f = x - (double)i;
      return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
    };
    out->latency_p50_ms = pct(0.50);
    out->latency_p99_ms = pct(0.99);
    out->latency_max_ms = v.back();
  }
  if (s->completed > 0) out->wall_ms = ms_since(s->t_first_submit, s->t_last_done);
  out->peak_inflight = s->peak_inflight;
  // sweep over the device intervals: +1 at a start, -1 at an end (ends
  // first at equal times, so touching intervals do not count as overlap)
  std::vector<std::pair<double, int>> ev;
  ev.reserve(2 * s->intervals.size());
  for (const auto& iv : s->intervals) {
    ev.emplace_back(iv.first, +1);
    ev.emplace_back(iv.second, -1);
  }
  std::sort(ev.begin(), ev.end());
  int64_t level = 0;
  double last = 0.0;
  for (const auto& e : ev) {
    if (level >= 2) out->overlap_ms += e.first - last;
    level += e.second;
    last = e.first;
    out->peak_concurrent = std::max(out->peak_concurrent, level);
  }
  return ESP_OK;
}

esp_status esp_server_reset_stats(esp_server_t s) {
  if (!s) return sfail(ESP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->completed = s->failed = 0;
  s->atoms_done = 0;
  s->latencies.clear();
  s->intervals.clear();
  s->peak_inflight = 0;
  s->any_submit = false;
  return ESP_OK;
}

esp_status esp_server_destroy(esp_server_t s) {
  if (!s) return ESP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->opts.device);
  for (Request* r : s->running) cudaEventSynchronize(r->ev);
  for (Request* r : s->late) cudaEventSynchronize(r->ev);
  for (auto& kv : s->plans) esp_destroy(kv.second->plan);
  for (auto& kv : s->tickets) {
    s->pinned.put(kv.second->buf, kv.second->cls);
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (kv.second->ev_start) cudaEventDestroy(kv.second->ev_start);
  }
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  cudaSetDevice(prev);
  delete s;
  return ESP_OK;
}

}  // extern "C"
