// fdlbm_server.cu -- continuous-batching serving runtime for FDLBM solves on one GPU.
//
// A worker thread owns all device work. Client threads submit requests (a solve: configuration,
// initial macros, step count), poll or wait for them, and collect results. Each round the worker:
//   1. admits queued requests in submission order while the HBM budget and the slots allow
//      (a request that does not fit waits at the head of the queue);
//   2. advances every admitted solve by the same k steps (k = min(round, fewest remaining)),
//      one batch per group of solves sharing scheme constants and precision: one kernel launch
//      per time step over all of the group's solves (fdlbm_batch_step);
//   3. retires finished solves (moments read back to host memory) and failed ones (a numerical
//      failure is reported; an FP32-storage solve is never re-run in FP64);
//   4. records each request's time to solution, from submission to retirement.
// The engine behind the scheduler is an interface: the GPU engine does the work above; the
// simulated engine touches no device and lets the scheduling policy be tested without a GPU.
#include <cuda_runtime.h>

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
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/fdlbm.h"
#include "fdlbm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  long long id = 0;
  fdlbm_config cfg;
  double bstate[4][4];
  long steps = 0;
  long sim_fail_step = 0;
  std::vector<double> init;  // rho, u, v, T (4 * nx * ny), released after admission
  size_t nbytes = 0;
  int status = FDLBM_REQ_QUEUED;
  long done = 0;
  fdlbm_t h = nullptr;
  fdlbm_batch_t batch = nullptr;
  Clock::time_point submitted, finished;
  std::vector<double> result;  // rho, u, v, T
  std::string error;
  int code = FDLBM_OK;  // error code of a failed request
  long remaining() const { return steps - done; }
};
using ReqPtr = std::shared_ptr<Req>;

struct Engine {
  virtual ~Engine() {}
  virtual size_t nbytes(const Req& r) = 0;
  virtual int create(Req& r, std::string* err) = 0;
  // advance every request by k steps; failed[i] = 1 for requests that hit a numerical failure
  virtual int step_all(std::vector<ReqPtr>& act, long k, std::vector<int>& failed, std::string* err) = 0;
  virtual int result(Req& r, std::string* err) = 0;
  virtual void release(Req& r) = 0;
};

// Real engine: one handle per request (library-owned device memory), one batch per scheme group.
struct GpuEngine : Engine {
  cudaStream_t stream = nullptr;
  bool separate = false;  // baseline: every solve stepped with its own launches, no batches
  std::map<std::tuple<double, double, double, double, double, int, int>, fdlbm_batch_t> batches;
  std::map<fdlbm_batch_t, int> tuned_size;  // members when the batch's tile was last autotuned
  GpuEngine(cudaStream_t s, bool sep) : stream(s), separate(sep) {}
  // The batch's tile variant from the autotuner (trial launches on the members' current states,
  // which do not advance them), when the batch is first stepped and again whenever its membership
  // has doubled or halved since.
  int tune(fdlbm_batch_t b, std::string* err) {
    const int n = fdlbm_batch_size(b);
    auto it = tuned_size.find(b);
    if (n < 1 || (it != tuned_size.end() && n < 2 * it->second && 2 * n > it->second)) return FDLBM_OK;
    const int rc = fdlbm_batch_autotune(b, 2, nullptr);
    if (rc) {
      *err = fdlbm_batch_last_error(b);
      return rc;
    }
    tuned_size[b] = n;
    return FDLBM_OK;
  }
  ~GpuEngine() override {
    for (auto& kv : batches) fdlbm_batch_destroy(kv.second);
  }
  size_t nbytes(const Req& r) override { return fdlbm_device_bytes(&r.cfg); }
  int create(Req& r, std::string* err) override {
    fdlbm_t h = nullptr;
    int rc = fdlbm_create_ex(&h, &r.cfg, nullptr, 0, stream);
    if (rc) {
      *err = fdlbm_last_error(nullptr);
      return rc;
    }
    for (int s = 0; s < 4 && !rc; ++s)
      if (r.cfg.bc[s] == FDLBM_BC_DIRICHLET)
        rc = fdlbm_set_boundary_state(h, s, r.bstate[s][0], r.bstate[s][1], r.bstate[s][2], r.bstate[s][3]);
    const size_t n = (size_t)r.cfg.nx * r.cfg.ny;
    if (!rc) rc = fdlbm_set_macro(h, r.init.data(), r.init.data() + n, r.init.data() + 2 * n, r.init.data() + 3 * n);
    const auto key = std::make_tuple(r.cfg.dx, r.cfg.dy, r.cfg.dt, r.cfg.tau, r.cfg.lambda, r.cfg.flags, r.cfg.prec);
    if (!rc && !separate) {
      auto it = batches.find(key);
      if (it == batches.end()) {
        fdlbm_batch_t b = nullptr;
        rc = fdlbm_batch_create(&b, stream);
        if (!rc) it = batches.emplace(key, b).first;
      }
      if (!rc) {
        rc = fdlbm_batch_add(it->second, h);
        if (!rc) r.batch = it->second;
      }
    }
    if (rc) {
      *err = fdlbm_last_error(h);
      fdlbm_destroy(h);
      return rc;
    }
    r.h = h;
    std::vector<double>().swap(r.init);
    return FDLBM_OK;
  }
  int step_all(std::vector<ReqPtr>& act, long k, std::vector<int>& failed, std::string* err) override {
    failed.assign(act.size(), 0);
    if (separate) {
      for (auto& r : act) {
        int rc = fdlbm_step(r->h, k);
        if (rc && rc != FDLBM_E_NUMERIC) {
          *err = fdlbm_last_error(r->h);
          return rc;
        }
      }
      for (size_t i = 0; i < act.size(); ++i)
        if (fdlbm_sync(act[i]->h) == FDLBM_E_NUMERIC) failed[i] = 1;
      return FDLBM_OK;
    }
    for (auto& kv : batches) {
      if (fdlbm_batch_size(kv.second) <= 0) continue;
      int rc = tune(kv.second, err);
      if (rc) return rc;
      rc = fdlbm_batch_step(kv.second, k);
      if (rc) {
        *err = fdlbm_batch_last_error(kv.second);
        return rc;
      }
    }
    int nfail = 0;
    for (auto& kv : batches) {
      if (fdlbm_batch_size(kv.second) <= 0) continue;
      int rc = fdlbm_batch_sync(kv.second, nullptr);
      if (rc < 0) {
        *err = fdlbm_batch_last_error(kv.second);
        return rc;
      }
      nfail += rc;
    }
    if (nfail)
      for (size_t i = 0; i < act.size(); ++i)
        if (fdlbm_sync(act[i]->h) == FDLBM_E_NUMERIC) failed[i] = 1;
    return FDLBM_OK;
  }
  int result(Req& r, std::string* err) override {
    const size_t n = (size_t)r.cfg.nx * r.cfg.ny;
    r.result.resize(4 * n);
    if (r.batch) {
      fdlbm_batch_remove(r.batch, r.h);
      r.batch = nullptr;
    }
    int rc = fdlbm_get_macro(r.h, r.result.data(), r.result.data() + n, r.result.data() + 2 * n, r.result.data() + 3 * n);
    if (rc) *err = fdlbm_last_error(r.h);
    return rc;
  }
  void release(Req& r) override {
    if (r.batch) fdlbm_batch_remove(r.batch, r.h);
    r.batch = nullptr;
    if (r.h) fdlbm_destroy(r.h);
    r.h = nullptr;
  }
};

// Simulated engine: no device work. A step of a solve "costs" ns_per_lup per site (a sleep of the
// whole round), a request fails when it reaches sim_fail_step, and its result is rho = u = v = T =
// the steps it took. For testing the scheduling policy on machines without a GPU.
struct SimEngine : Engine {
  double ns_per_lup;
  explicit SimEngine(double ns) : ns_per_lup(ns) {}
  size_t nbytes(const Req& r) override { return fdlbm_device_bytes(&r.cfg); }
  int create(Req& r, std::string*) override {
    std::vector<double>().swap(r.init);
    return FDLBM_OK;
  }
  int step_all(std::vector<ReqPtr>& act, long k, std::vector<int>& failed, std::string*) override {
    failed.assign(act.size(), 0);
    double sites = 0;
    for (size_t i = 0; i < act.size(); ++i) {
      sites += (double)act[i]->cfg.nx * act[i]->cfg.ny;
      const long f = act[i]->sim_fail_step;
      if (f > 0 && act[i]->done < f && act[i]->done + k >= f) failed[i] = 1;
    }
    std::this_thread::sleep_for(std::chrono::nanoseconds((long long)(ns_per_lup * sites * k)));
    return FDLBM_OK;
  }
  int result(Req& r, std::string*) override {
    r.result.assign(4 * (size_t)r.cfg.nx * r.cfg.ny, (double)r.done);
    return FDLBM_OK;
  }
  void release(Req&) override {}
};

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

}  // namespace

struct fdlbm_server_ctx {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  size_t budget = 0;
  int max_slots = 0;
  long round_steps = 0;
  std::unique_ptr<Engine> eng;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::deque<ReqPtr> queue;
  std::vector<ReqPtr> active;  // worker thread only
  std::unordered_map<long long, ReqPtr> table;
  long long next_id = 1;
  size_t used = 0;
  // statistics
  std::vector<double> latencies;
  double lups = 0;
  bool started = false;
  Clock::time_point t_first, t_last;
  long long rounds = 0, n_submitted = 0, n_failed = 0, n_done = 0;
  int max_active = 0;
  size_t max_bytes = 0;
  std::string err;
};

namespace {

int sfail(fdlbm_server_ctx* s, int code, const std::string& msg) {
  if (s) {
    std::lock_guard<std::mutex> g(s->mu);
    s->err = msg;
  } else {
    fdlbm::set_thread_error(msg.c_str());
  }
  return code;
}

void retire(fdlbm_server_ctx* s, const ReqPtr& r, bool failed, const std::string& why, int code = FDLBM_E_NUMERIC) {
  // called with s->mu held
  r->finished = Clock::now();
  s->t_last = r->finished;
  s->used -= r->nbytes;
  if (failed) {
    r->status = FDLBM_REQ_FAILED;
    r->error = why;
    r->code = code;
    ++s->n_failed;
  } else {
    r->status = FDLBM_REQ_DONE;
    ++s->n_done;
    s->latencies.push_back(seconds(r->finished - r->submitted));
  }
}

void worker_main(fdlbm_server_ctx* s, bool gpu) {
  if (gpu) cudaSetDevice(s->device);
  for (;;) {
    std::vector<ReqPtr> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty() || !s->active.empty(); });
      if (s->stop) break;
      size_t used = s->used;
      int slots = (int)s->active.size();
      while (!s->queue.empty() && slots < s->max_slots && used + s->queue.front()->nbytes <= s->budget) {
        ReqPtr r = s->queue.front();
        s->queue.pop_front();
        used += r->nbytes;
        ++slots;
        r->status = FDLBM_REQ_ACTIVE;
        admit.push_back(r);
      }
      s->used = used;
    }
    for (auto& r : admit) {  // device work outside the lock
      std::string err;
      int rc = s->eng->create(*r, &err);
      std::lock_guard<std::mutex> g(s->mu);
      if (rc) {
        retire(s, r, true, "admission failed: " + err, rc);
        s->cv_done.notify_all();
      } else {
        s->active.push_back(r);
      }
    }
    if (s->active.empty()) continue;
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->max_active = std::max(s->max_active, (int)s->active.size());
      s->max_bytes = std::max(s->max_bytes, s->used);
    }
    long k = s->round_steps;
    for (auto& r : s->active) k = std::min(k, r->remaining());
    std::vector<int> failed;
    std::string err;
    int rc = s->eng->step_all(s->active, k, failed, &err);
    std::vector<ReqPtr> keep;
    struct Out {
      ReqPtr r;
      std::string why;
      int code;
    };
    std::vector<Out> done_list;
    for (size_t i = 0; i < s->active.size(); ++i) {
      ReqPtr& r = s->active[i];
      if (rc) {
        done_list.push_back({r, "engine failure: " + err, rc});
        continue;
      }
      r->done += k;
      if (failed[i]) {
        done_list.push_back({r, "numerical failure (non-finite moments, n <= 0 or T <= 0)", FDLBM_E_NUMERIC});
      } else if (r->remaining() <= 0) {
        std::string e2;
        int rr = s->eng->result(*r, &e2);
        done_list.push_back({r, rr ? ("result read-back failed: " + e2) : std::string(), rr});
      } else {
        keep.push_back(r);
      }
    }
    for (auto& d : done_list) s->eng->release(*d.r);
    {
      std::lock_guard<std::mutex> g(s->mu);
      double sites = 0;
      for (auto& r : s->active) sites += (double)r->cfg.nx * r->cfg.ny;
      if (!rc) s->lups += sites * (double)k;
      ++s->rounds;
      for (auto& d : done_list) retire(s, d.r, !d.why.empty(), d.why, d.code);
    }
    s->active.swap(keep);
    s->cv_done.notify_all();
  }
  // shutting down: release what is still on the device; queued and active requests are cancelled
  for (auto& r : s->active) s->eng->release(*r);
  std::lock_guard<std::mutex> g(s->mu);
  for (auto& r : s->active) {
    r->status = FDLBM_REQ_CANCELLED;
    s->used -= r->nbytes;
  }
  for (auto& r : s->queue) r->status = FDLBM_REQ_CANCELLED;
  s->active.clear();
  s->queue.clear();
  s->cv_done.notify_all();
}

}  // namespace

extern "C" {

int fdlbm_server_create(fdlbm_server_t* out, size_t budget_bytes, int max_slots, long round_steps, int engine,
                        void* cuda_stream) {
  if (!out) return sfail(nullptr, FDLBM_E_ARG, "out is NULL");
  *out = nullptr;
  if (budget_bytes == 0 || max_slots < 1 || round_steps < 1)
    return sfail(nullptr, FDLBM_E_ARG, "budget_bytes, max_slots and round_steps must be positive");
  if (engine != FDLBM_ENGINE_GPU && engine != FDLBM_ENGINE_SIMULATED && engine != FDLBM_ENGINE_GPU_SEPARATE)
    return sfail(nullptr, FDLBM_E_ARG, "unknown engine");
  const bool gpu = engine != FDLBM_ENGINE_SIMULATED;
  fdlbm_server_ctx* s = new (std::nothrow) fdlbm_server_ctx();
  if (!s) return sfail(nullptr, FDLBM_E_OOM, "host allocation failed");
  s->budget = budget_bytes;
  s->max_slots = max_slots;
  s->round_steps = round_steps;
  if (gpu) {
    cudaError_t e = cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    if (e == cudaSuccess && !s->stream) {
      e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
      s->own_stream = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
      delete s;
      return sfail(nullptr, FDLBM_E_CUDA, std::string("server stream: ") + cudaGetErrorString(e));
    }
    s->eng.reset(new GpuEngine(s->stream, engine == FDLBM_ENGINE_GPU_SEPARATE));
  } else {
    s->eng.reset(new SimEngine(1.0));
  }
  s->worker = std::thread(worker_main, s, gpu);
  *out = s;
  return FDLBM_OK;
}

int fdlbm_server_submit(fdlbm_server_t s, const fdlbm_request* req, long long* id) {
  if (!s || !req || !id) return sfail(s, FDLBM_E_ARG, "server, request or id is NULL");
  std::string why;
  if (!fdlbm::valid_cfg(&req->cfg, &why)) return sfail(s, FDLBM_E_ARG, why);
  if (req->steps < 0) return sfail(s, FDLBM_E_ARG, "steps < 0");
  if (!req->rho || !req->u || !req->v || !req->T) return sfail(s, FDLBM_E_ARG, "NULL initial macro array");
  ReqPtr r = std::make_shared<Req>();
  r->cfg = req->cfg;
  std::memcpy(r->bstate, req->bstate, sizeof(r->bstate));
  r->steps = req->steps;
  r->sim_fail_step = req->sim_fail_step;
  const size_t n = (size_t)req->cfg.nx * req->cfg.ny;
  r->init.resize(4 * n);
  std::memcpy(r->init.data(), req->rho, n * sizeof(double));
  std::memcpy(r->init.data() + n, req->u, n * sizeof(double));
  std::memcpy(r->init.data() + 2 * n, req->v, n * sizeof(double));
  std::memcpy(r->init.data() + 3 * n, req->T, n * sizeof(double));
  r->nbytes = s->eng->nbytes(*r);
  std::lock_guard<std::mutex> g(s->mu);
  r->id = s->next_id++;
  r->submitted = Clock::now();
  if (!s->started) {
    s->started = true;
    s->t_first = r->submitted;
  }
  ++s->n_submitted;
  s->table[r->id] = r;
  if (r->nbytes > s->budget) {
    r->status = FDLBM_REQ_FAILED;
    r->error = "the solve needs more device memory than the server's budget";
    r->code = FDLBM_E_OOM;
    r->finished = r->submitted;
    ++s->n_failed;
    s->cv_done.notify_all();
  } else {
    s->queue.push_back(r);
    s->cv_work.notify_one();
  }
  *id = r->id;
  return FDLBM_OK;
}

int fdlbm_server_poll(fdlbm_server_t s, long long id, int* status) {
  if (!s || !status) return sfail(s, FDLBM_E_ARG, "server or status is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return FDLBM_E_ARG;
  *status = it->second->status;
  return FDLBM_OK;
}

int fdlbm_server_wait(fdlbm_server_t s, long long id, double timeout_s, int* status) {
  if (!s) return sfail(s, FDLBM_E_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return FDLBM_E_ARG;
  ReqPtr r = it->second;
  auto pred = [&] { return r->status >= FDLBM_REQ_DONE; };
  bool ok = timeout_s < 0 ? (s->cv_done.wait(lk, pred), true)
                          : s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
  if (status) *status = r->status;
  return ok ? FDLBM_OK : FDLBM_E_TIMEOUT;
}

int fdlbm_server_result(fdlbm_server_t s, long long id, double* rho, double* u, double* v, double* T,
                        double* seconds_to_solution) {
  if (!s) return sfail(s, FDLBM_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return FDLBM_E_ARG;
  ReqPtr r = it->second;
  if (r->status == FDLBM_REQ_FAILED || r->status == FDLBM_REQ_CANCELLED) {
    s->err = r->status == FDLBM_REQ_CANCELLED ? std::string("cancelled") : r->error;
    const int code = r->status == FDLBM_REQ_CANCELLED ? FDLBM_E_STATE : r->code;
    s->table.erase(it);
    return code;
  }
  if (r->status != FDLBM_REQ_DONE) return FDLBM_E_STATE;
  const size_t n = (size_t)r->cfg.nx * r->cfg.ny;
  double* dst[4] = {rho, u, v, T};
  for (int a = 0; a < 4; ++a)
    if (dst[a]) std::memcpy(dst[a], r->result.data() + a * n, n * sizeof(double));
  if (seconds_to_solution) *seconds_to_solution = seconds(r->finished - r->submitted);
  s->table.erase(it);
  return FDLBM_OK;
}

int fdlbm_server_stats(fdlbm_server_t s, fdlbm_server_stats_t* st) {
  if (!s || !st) return sfail(s, FDLBM_E_ARG, "server or stats is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->n_submitted;
  st->done = s->n_done;
  st->failed = s->n_failed;
  st->queued = (long long)s->queue.size();
  st->rounds = s->rounds;
  st->max_active = s->max_active;
  st->max_bytes = s->max_bytes;
  std::vector<double> lat = s->latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double p) {
    if (lat.empty()) return 0.0;
    const double pos = p / 100.0 * (lat.size() - 1);
    const size_t i = (size_t)pos;
    const double fr = pos - i;
    return i + 1 < lat.size() ? lat[i] * (1 - fr) + lat[i + 1] * fr : lat[i];
  };
  st->p50_s = pct(50);
  st->p99_s = pct(99);
  double sum = 0;
  for (double x : lat) sum += x;
  st->mean_s = lat.empty() ? 0.0 : sum / lat.size();
  st->wall_s = s->started ? seconds(s->t_last - s->t_first) : 0.0;
  st->aggregate_glups = st->wall_s > 0 ? s->lups / st->wall_s / 1e9 : 0.0;
  return FDLBM_OK;
}

int fdlbm_server_destroy(fdlbm_server_t s) {
  if (!s) return FDLBM_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  s->eng.reset();
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return FDLBM_OK;
}

const char* fdlbm_server_last_error(fdlbm_server_t s) {
  if (!s) return fdlbm_last_error(nullptr);
  std::lock_guard<std::mutex> g(s->mu);
  return s->err.c_str();
}

}  // extern "C"
