// serve.cu -- continuous-batching request loop over resident plans
// (csfmm_server_* in include/csfmm.h).
//
// One scheduler thread owns every plan, workspace and slot.  Callers only
// append requests to a queue under the mutex and wait on a condition
// variable.  The scheduler (1) retires finished slots by polling their CUDA
// events, (2) admits requests while a slot is free and the device memory the
// request needs fits in the budget (evicting idle cached plans, least
// recently used first), and (3) sleeps briefly when nothing changed.
// Admission order (csfmm_server_set_policy): first come first served, or
// (default) the cheapest pending request first -- cost estimated from its
// points, right-hand sides and proxies -- with two guards: a request that
// has waited longer than the aging bound goes first regardless of its cost
// (and nothing is admitted past it while it does not fit), and large
// requests (at least 2^20 points) hold at most half of the slots, so that a
// burst of large requests cannot block small ones behind them.  Under that
// policy a small request also runs on its slot's high-priority stream with
// every pass on that stream (its plan is built with CSFMM_SCHED_NO_OVERLAP),
// so the block scheduler serves its kernels before pending blocks of large
// requests instead of letting them queue behind those.
// Each admitted request runs on its slot's stream with its own workspace, so
// requests of different sizes and kernels overlap on the GPU; a request's
// result does not depend on what else runs (deterministic kernels, private
// workspace, read-only shared plan).
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "csfmm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct PlanKey {
  uint64_t key;
  int kid, degree, N0, prec;
  double theta;
  bool operator<(const PlanKey &o) const {
    if (key != o.key) return key < o.key;
    if (kid != o.kid) return kid < o.kid;
    if (degree != o.degree) return degree < o.degree;
    if (N0 != o.N0) return N0 < o.N0;
    if (prec != o.prec) return prec < o.prec;
    return theta < o.theta;
  }
};

struct CachedPlan {
  csfmm_plan plan = nullptr;
  int64_t bytes = 0;                      // plan + its default workspace
  bool default_ws_free = true;            // the plan's own workspace (csfmm_evaluate)
  std::vector<csfmm_workspace> idle_ws;   // extra workspaces (csfmm_evaluate_ws)
  std::vector<csfmm_workspace> all_ws;
  int64_t ws_bytes = 0;                   // bytes of one extra workspace
  int in_flight = 0;
  uint64_t last_use = 0;
};

struct Request {
  csfmm_request r{};
  csfmm_request_timing t{};
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;     // default (lowest) priority
  cudaStream_t stream_hi = nullptr;  // highest priority: small requests under the size-aware policy
  cudaStream_t cur = nullptr;        // the stream of the request in flight
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int64_t req = -1;
  PlanKey key{};
  bool acquired = false;         // holds a workspace of plans[key] and counts as in flight
  csfmm_workspace ws = nullptr;  // nullptr: the plan's default workspace
};

int kdim(int k) { return k == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1; }

// Device bytes of one workspace for R right-hand sides (mirrors workspace_alloc).
int64_t workspace_bytes_estimate(int64_t N, int64_t cells, int64_t P, int64_t dim, int64_t real,
                                 int64_t R) {
  // FP32 form: single-precision weights and the symmetric near field's
  // cross-pair partials (one float per point and PP partner, ~36 partners)
  return R * N * 8 + (real == 4 ? R * N * 4 + 36 * N * 4 : 0) +
         cells * R * P * (real + 8 * dim) + R * N * dim * 8;
}

// Device bytes of a plan built with CSFMM_SERVER_MAX_NRHS right-hand sides
// (estimate used before the build; replaced by the plan's own count after).
int64_t estimate_plan_bytes(const csfmm_request &r) {
  const int64_t N = r.N, p = r.degree + 1, P = p * p, dim = kdim(r.kernel_id);
  const int64_t real = r.precision == CSFMM_FP64 ? 8 : 4;
  const int64_t R = CSFMM_SERVER_MAX_NRHS;
  const int64_t leaves = 4 * N / (r.max_leaf > 0 ? r.max_leaf : 1) + 6;
  const int64_t cells = (4 * leaves) / 3 + 6;
  int64_t b = N * (24 + 4 + 2 * p * real + 16 + 4);             // points, perm, L rows, offsets
  b += cells * (3 * P * 12 + 160 + 8 * 64);                      // geometry, proxies, lists
  b += workspace_bytes_estimate(N, cells, P, dim, real, R);      // default workspace
  return b;
}

}  // namespace

// Relative cost of a request (points x (right-hand sides + a fixed part) x
// proxies), used only to order admissions.
double request_cost(const csfmm_request &r) {
  const double p = r.degree + 1;
  return (double)r.N * (4.0 + r.nrhs) * p * p;
}
constexpr int64_t kLargeRequestN = 1 << 20;

struct csfmm_server_s {
  int device = 0;
  int64_t budget = 0;
  int policy = CSFMM_SERVE_CHEAPEST_FIRST;
  double age_ms = 250.0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<int64_t> pending;
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_id = 0;
  std::map<PlanKey, CachedPlan> plans;
  csfmm_server_stats st{};
  uint64_t use_clock = 0;
  bool stop = false;
  cudaStream_t build_stream = nullptr;
  Clock::time_point t0;
  std::thread th;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  int in_flight() const {
    int n = 0;
    for (const Slot &s : slots) n += s.req >= 0;
    return n;
  }
  void run();
  bool retire();
  bool admit(std::unique_lock<std::mutex> &lk);
  // Index into `pending` of the next request to admit, or -1 to wait.
  int pick(double now);
  void finish(Slot &s, int status);
};

void csfmm_server_s::finish(Slot &s, int status) {
  Request &q = reqs[s.req];
  float ms = 0.f;
  if (status == CSFMM_OK && cudaEventElapsedTime(&ms, s.e0, s.e1) != cudaSuccess) cudaGetLastError();
  q.t.gpu_ms = ms;
  q.t.done_ms = now_ms();
  q.t.status = status;
  q.done = true;
  auto it = plans.find(s.key);
  if (s.acquired && it != plans.end()) {
    CachedPlan &cp = it->second;
    if (s.ws) cp.idle_ws.push_back(s.ws);
    else cp.default_ws_free = true;
    cp.in_flight--;
  }
  s.acquired = false;
  if (status == CSFMM_OK) st.completed++;
  else st.failed++;
  s.req = -1;
  s.ws = nullptr;
  cv_done.notify_all();
}

bool csfmm_server_s::retire() {
  bool any = false;
  for (Slot &s : slots) {
    if (s.req < 0) continue;
    cudaError_t e = cudaEventQuery(s.e1);
    if (e == cudaErrorNotReady) continue;
    int status = CSFMM_OK;
    if (e != cudaSuccess) {
      cudaGetLastError();
      status = CSFMM_ERR_CUDA;
    } else if (csfmm_plan_sync(plans[s.key].plan, s.cur) != CSFMM_OK) {
      status = CSFMM_ERR_DEVICE;
    }
    finish(s, status);
    any = true;
  }
  return any;
}

int csfmm_server_s::pick(double now) {
  if (pending.empty()) return -1;
  if (policy == CSFMM_SERVE_FIFO) return 0;
  // an aged request goes first (pending is in submission order)
  if (now - reqs[pending.front()].t.submit_ms > age_ms) return 0;
  int large = 0;
  for (const Slot &sl : slots)
    if (sl.req >= 0 && reqs[sl.req].r.N >= kLargeRequestN) ++large;
  const int large_cap = (int)slots.size() / 2 > 0 ? (int)slots.size() / 2 : 1;
  int best = -1;
  double best_cost = 0.0;
  for (size_t k = 0; k < pending.size(); ++k) {
    const csfmm_request &r = reqs[pending[k]].r;
    if (r.N >= kLargeRequestN && large >= large_cap) continue;
    const double c = request_cost(r);
    if (best < 0 || c < best_cost) {
      best = (int)k;
      best_cost = c;
    }
  }
  return best;
}

bool csfmm_server_s::admit(std::unique_lock<std::mutex> &lk) {
  bool any = false;
  while (!pending.empty()) {
    int si = -1;
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i].req < 0) { si = (int)i; break; }
    if (si < 0) break;
    const int pk = pick(now_ms());
    if (pk < 0) break;
    const int64_t id = pending[pk];
    Request &q = reqs[id];
    const csfmm_request &r = q.r;
    PlanKey key{r.plan_key, r.kernel_id, r.degree, r.max_leaf, r.precision, r.theta};
    auto it = plans.find(key);
    int64_t need = 0;
    if (it == plans.end()) {
      need = estimate_plan_bytes(r);
    } else if (!it->second.default_ws_free && it->second.idle_ws.empty()) {
      need = it->second.ws_bytes;
    }
    // evict idle plans (least recently used first) until the request fits
    while (st.bytes_held + need > budget) {
      auto victim = plans.end();
      for (auto p = plans.begin(); p != plans.end(); ++p) {
        const bool same = !(p->first < key) && !(key < p->first);
        if (p->second.in_flight == 0 && !same &&
            (victim == plans.end() || p->second.last_use < victim->second.last_use))
          victim = p;
      }
      if (victim == plans.end()) break;
      for (csfmm_workspace w : victim->second.all_ws) csfmm_workspace_destroy(w);
      csfmm_plan_destroy(victim->second.plan);
      st.bytes_held -= victim->second.bytes + victim->second.ws_bytes * (int64_t)victim->second.all_ws.size();
      st.plans_evicted++;
      plans.erase(victim);
      it = plans.find(key);
    }
    if (st.bytes_held + need > budget) break;  // wait for running requests to finish
    pending.erase(pending.begin() + pk);
    Slot &s = slots[si];
    s.req = id;
    s.key = key;
    q.t.slot = si;
    csfmm_status status = CSFMM_OK;
    lk.unlock();  // CUDA work below; only this thread touches plans and slots
    if (it == plans.end()) {
      csfmm_options opt{};
      opt.precision = r.precision;
      opt.max_nrhs = CSFMM_SERVER_MAX_NRHS;
      opt.use_graphs = 1;
      if (policy == CSFMM_SERVE_CHEAPEST_FIRST && r.N < kLargeRequestN)
        opt.schedule = CSFMM_SCHED_NO_OVERLAP;
      csfmm_plan h = nullptr;
      status = csfmm_plan_create(r.points, r.N, r.kernel_id, r.degree, r.theta, r.max_leaf, &opt,
                                 build_stream, &h);
      if (status == CSFMM_OK) {
        CachedPlan cp;
        cp.plan = h;
        cp.bytes = h->impl.stats.device_bytes;
        const csfmm::Plan &pl = h->impl;
        cp.ws_bytes = workspace_bytes_estimate(pl.N, pl.ncells, pl.P, pl.dim,
                                               pl.precision == CSFMM_FP64 ? 8 : 4,
                                               CSFMM_SERVER_MAX_NRHS);
        lk.lock();
        it = plans.emplace(key, cp).first;
        st.bytes_held += cp.bytes;
        st.plans_built++;
        q.t.built_plan = 1;
        lk.unlock();
      }
    }
    if (status == CSFMM_OK) {
      CachedPlan &cp = it->second;
      if (cp.default_ws_free) {
        cp.default_ws_free = false;
        s.ws = nullptr;
      } else if (!cp.idle_ws.empty()) {
        s.ws = cp.idle_ws.back();
        cp.idle_ws.pop_back();
      } else {
        csfmm_workspace w = nullptr;
        status = csfmm_workspace_create(cp.plan, CSFMM_SERVER_MAX_NRHS, &w);
        if (status == CSFMM_OK) {
          cp.all_ws.push_back(w);
          s.ws = w;
          lk.lock();
          st.bytes_held += w->impl.arena.bytes;
          cp.ws_bytes = w->impl.arena.bytes;
          lk.unlock();
        }
      }
      if (status == CSFMM_OK) {
        cp.in_flight++;
        s.acquired = true;
        cp.last_use = ++use_clock;
        q.t.admit_ms = now_ms();
        s.cur = (policy == CSFMM_SERVE_CHEAPEST_FIRST && r.N < kLargeRequestN) ? s.stream_hi
                                                                               : s.stream;
        cudaEventRecord(s.e0, s.cur);
        if (s.ws)
          status = csfmm_evaluate_ws(cp.plan, s.ws, r.weights, r.nrhs, r.out, s.cur);
        else
          status = csfmm_evaluate(cp.plan, r.weights, r.nrhs, r.out, s.cur);
        cudaEventRecord(s.e1, s.cur);
      }
    }
    lk.lock();
    if (st.bytes_held > st.peak_bytes_held) st.peak_bytes_held = st.bytes_held;
    const int inf = in_flight();
    if (inf > st.max_in_flight) st.max_in_flight = inf;
    if (status != CSFMM_OK) {
      cudaStreamSynchronize(s.cur ? s.cur : s.stream);
      finish(s, status);
    }
    any = true;
  }
  return any;
}

void csfmm_server_s::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool changed = retire();
    changed |= admit(lk);
    if (stop && pending.empty() && in_flight() == 0) break;
    if (!changed) cv_sched.wait_for(lk, std::chrono::microseconds(50));
  }
}

using namespace csfmm;

extern "C" {

csfmm_status csfmm_server_create(int64_t hbm_budget_bytes, int slots, csfmm_server *out) {
  if (!out || slots < 1 || slots > 64 || hbm_budget_bytes <= 0) {
    set_error("out must be non-NULL, 1 <= slots <= 64 and the budget positive");
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  csfmm_server s = new (std::nothrow) csfmm_server_s;
  if (!s) {
    set_error("host allocation failed");
    return CSFMM_ERR_OUT_OF_MEMORY;
  }
  cudaGetDevice(&s->device);
  s->budget = hbm_budget_bytes;
  s->st.budget_bytes = hbm_budget_bytes;
  s->st.slots = slots;
  s->slots.resize(slots);
  cudaError_t e = cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking);
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  for (Slot &sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.e1);
  }
  if (e != cudaSuccess) {
    csfmm_status st = cuda_status(e, "server stream/event creation");
    for (Slot &sl : s->slots) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.stream_hi) cudaStreamDestroy(sl.stream_hi);
      if (sl.e0) cudaEventDestroy(sl.e0);
      if (sl.e1) cudaEventDestroy(sl.e1);
    }
    if (s->build_stream) cudaStreamDestroy(s->build_stream);
    delete s;
    return st;
  }
  s->t0 = Clock::now();
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return CSFMM_OK;
}

csfmm_status csfmm_server_set_policy(csfmm_server s, int policy, double age_ms) {
  if (!s || (policy != CSFMM_SERVE_FIFO && policy != CSFMM_SERVE_CHEAPEST_FIRST) ||
      !(age_ms > 0.0)) {
    set_error("server must be non-NULL, policy CSFMM_SERVE_FIFO or CSFMM_SERVE_CHEAPEST_FIRST "
              "and age_ms > 0");
    return CSFMM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->policy = policy;
  s->age_ms = age_ms;
  return CSFMM_OK;
}

csfmm_status csfmm_server_submit(csfmm_server s, const csfmm_request *req, int64_t *id) {
  if (!s || !req || !id) {
    set_error("server, request and id must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  const csfmm_request &r = *req;
  if (!r.points || !r.weights || !r.out || r.N < 1 || r.nrhs < 1 ||
      r.nrhs > CSFMM_SERVER_MAX_NRHS || r.degree < 1 || r.degree > kMaxDegree ||
      !(r.theta > 0.0 && r.theta < 1.0) || r.max_leaf < 1 ||
      (r.precision != CSFMM_FP64 && r.precision != CSFMM_FP32_BULK) ||
      (r.kernel_id != CSFMM_KERNEL_LAPLACE && r.kernel_id != CSFMM_KERNEL_BIOT_SAVART &&
       r.kernel_id != CSFMM_KERNEL_NEWTON && r.kernel_id != CSFMM_KERNEL_BIHARMONIC &&
       r.kernel_id != CSFMM_KERNEL_SAL &&
       r.kernel_id != CSFMM_KERNEL_ONE)) {
    set_error("invalid request");
    return CSFMM_ERR_INVALID_ARG;
  }
  if (estimate_plan_bytes(r) > s->budget) {
    set_error("the request's plan (about %lld bytes) can never fit the budget of %lld bytes",
              (long long)estimate_plan_bytes(r), (long long)s->budget);
    return CSFMM_ERR_OUT_OF_MEMORY;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t k = s->next_id++;
  Request q;
  q.r = r;
  q.t.submit_ms = s->now_ms();
  q.t.slot = -1;
  s->reqs.emplace(k, q);
  s->pending.push_back(k);
  s->st.submitted++;
  *id = k;
  s->cv_sched.notify_one();
  return CSFMM_OK;
}

csfmm_status csfmm_server_poll(csfmm_server s, int64_t id, int *done, csfmm_request_timing *t) {
  if (!s || !done) {
    set_error("server and done must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_error("unknown request id %lld", (long long)id);
    return CSFMM_ERR_INVALID_ARG;
  }
  *done = it->second.done;
  if (t) *t = it->second.t;
  return CSFMM_OK;
}

csfmm_status csfmm_server_wait(csfmm_server s, int64_t id, csfmm_request_timing *t) {
  if (!s) {
    set_error("server is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    set_error("unknown request id %lld", (long long)id);
    return CSFMM_ERR_INVALID_ARG;
  }
  s->cv_done.wait(lk, [&] { return it->second.done; });
  if (t) *t = it->second.t;
  return (csfmm_status)it->second.t.status;
}

csfmm_status csfmm_server_drain(csfmm_server s) {
  if (!s) {
    set_error("server is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->pending.empty() && s->in_flight() == 0; });
  return s->st.failed ? CSFMM_ERR_DEVICE : CSFMM_OK;
}

csfmm_status csfmm_server_stats_get(csfmm_server s, csfmm_server_stats *out) {
  if (!s || !out) {
    set_error("server and stats must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return CSFMM_OK;
}

csfmm_status csfmm_server_destroy(csfmm_server s) {
  if (!s) return CSFMM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_sched.notify_one();
  }
  s->th.join();
  for (auto &kv : s->plans) {
    for (csfmm_workspace w : kv.second.all_ws) csfmm_workspace_destroy(w);
    csfmm_plan_destroy(kv.second.plan);
  }
  for (Slot &sl : s->slots) {
    cudaStreamDestroy(sl.stream);
    cudaStreamDestroy(sl.stream_hi);
    cudaEventDestroy(sl.e0);
    cudaEventDestroy(sl.e1);
  }
  cudaStreamDestroy(s->build_stream);
  delete s;
  return CSFMM_OK;
}

}  // extern "C"
