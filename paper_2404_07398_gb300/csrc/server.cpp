// Serving loop: a worker thread that keeps batched solvers (engines) busy with
// the columns of queued requests over resident prepared meshes.  Continuous
// batching happens inside the engines (columns join at step boundaries as
// lanes and memory free up); the worker launches one step on every busy
// engine before waiting for any of them, so engines on different streams run
// concurrently on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  ifilt_mesh mesh = nullptr;
  ifilt_solve_opts opts{};
  int32_t F = 0;
  const double* fields = nullptr;
  std::vector<double> k;
  double* out = nullptr;
  ifilt_col_stats* stats = nullptr;
  int columns = 0, done = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  int status = IFILT_OK;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// mesh, order, precision, n = 2 form, preconditioner, error tolerance, cycle
using Key = std::tuple<ifilt_mesh, int, int, int, int, double, int>;

struct EngineSlot {
  std::unique_ptr<ifilt::Engine> engine;
  cudaStream_t stream = nullptr;
  bool launched = false;
};

}  // namespace

struct ifilt_server_s {
  ifilt_server_opts opts{};
  int device = 0;
  int64_t budget = 0;
  Clock::time_point t0 = Clock::now();
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> incoming;
  std::map<int64_t, Request> reqs;
  int64_t next_id = 1;
  bool stopping = false;
  int failed = 0;  // negative status once the worker hit an error
  std::string error;
  std::map<Key, EngineSlot> engines;  // touched by the worker only
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // worker: turn new requests into engine columns
  void admit_new(std::vector<int64_t>& ids) {
    for (int64_t id : ids) {
      Request* r;
      {
        std::lock_guard<std::mutex> lk(mu);
        r = &reqs[id];
      }
      const ifilt::HostPrepared& h = r->mesh->host;
      ifilt_solve_opts o = r->opts;
      o.method = IFILT_METHOD_BATCHED;
      o.max_lanes = opts.max_lanes;
      o.check_every = opts.check_every;
      const bool cplx = ifilt::complex_form(o);
      Key key{r->mesh, o.order, o.precision, o.order >= 2 ? (cplx ? 2 : 1) : 0, o.precond, o.err_tol, o.mg_cycle};
      auto it = engines.find(key);
      if (it == engines.end()) {
        EngineSlot slot;
        IFILT_CUDA(cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking));
        slot.engine.reset(ifilt::make_engine(r->mesh, o, slot.stream, budget));
        it = engines.emplace(key, std::move(slot)).first;
      }
      const int nsys = h.placement == IFILT_CELL ? 2 : 1;
      const int K = (int)r->k.size();
      std::vector<ifilt::ColumnJob> jobs;
      for (int f = 0; f < r->F; f++)
        for (int s = 0; s < nsys; s++)
          for (int j = 0; j < K; j++) {
            ifilt::ColumnJob c;
            c.request = id;
            c.field = r->fields + (int64_t)f * h.n_comp * h.n_in;
            c.sys = s;
            c.k = r->k[j];
            c.out = r->out + ((int64_t)f * K + j) * h.n_comp * h.n_out;
            c.stat = r->stats ? &r->stats[((int64_t)f * K + j) * nsys + s] : nullptr;
            jobs.push_back(c);
          }
      std::stable_sort(jobs.begin(), jobs.end(), [](const ifilt::ColumnJob& a, const ifilt::ColumnJob& b) {
        return a.k < b.k;
      });
      it->second.engine->submit(jobs);
      std::lock_guard<std::mutex> lk(mu);
      r->columns = (int)jobs.size();
      r->state = 1;
      r->t_start = now();
    }
  }

  void finish_columns(const std::vector<ifilt::ColumnDone>& done) {
    std::lock_guard<std::mutex> lk(mu);
    bool any = false;
    for (const auto& d : done) {
      auto it = reqs.find(d.request);
      if (it == reqs.end()) continue;
      Request& r = it->second;
      r.done++;
      if (d.status != IFILT_OK) r.status = IFILT_NOT_CONVERGED;
      if (r.done == r.columns) {
        r.state = 2;
        r.t_done = now();
        any = true;
      }
    }
    if (any) cv_done.notify_all();
  }

  void fail_all(ifilt_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(mu);
    failed = st;
    error = msg;
    for (auto& kv : reqs)
      if (kv.second.state < 2) {
        kv.second.state = 3;
        kv.second.status = st;
        kv.second.t_done = now();
      }
    cv_done.notify_all();
  }

  void loop() {
    try {
      IFILT_CUDA(cudaSetDevice(device));
      while (true) {
        std::vector<int64_t> ids;
        {
          std::unique_lock<std::mutex> lk(mu);
          auto busy = [&] {
            for (auto& kv : engines)
              if (!kv.second.engine->idle()) return true;
            return false;
          };
          while (incoming.empty() && !busy() && !stopping) cv_work.wait_for(lk, std::chrono::milliseconds(50));
          if (stopping) {
            // cancel whatever has not finished; the engines are freed by destroy
            for (auto& kv : reqs)
              if (kv.second.state < 2) {
                kv.second.state = 3;
                kv.second.status = IFILT_EINVAL;
                kv.second.t_done = now();
              }
            cv_done.notify_all();
            return;
          }
          ids.assign(incoming.begin(), incoming.end());
          incoming.clear();
        }
        admit_new(ids);
        // memory: each engine may grow into what the others do not hold
        int64_t held = 0;
        for (auto& kv : engines) held += kv.second.engine->bytes_held();
        for (auto& kv : engines) {
          ifilt::Engine& e = *kv.second.engine;
          e.set_budget(std::max<int64_t>(budget - (held - e.bytes_held()), 1));
        }
        for (auto& kv : engines) {
          ifilt::Engine& e = *kv.second.engine;
          if (e.idle()) continue;
          e.launch();
          kv.second.launched = true;
        }
        std::vector<ifilt::ColumnDone> done;
        for (auto& kv : engines) {
          if (!kv.second.launched) continue;
          kv.second.launched = false;
          kv.second.engine->settle(done);
        }
        if (!done.empty()) finish_columns(done);
      }
    } catch (const ifilt::Error& e) {
      fail_all(e.status, e.msg);
    } catch (const std::exception& e) {
      fail_all(IFILT_ECUDA, e.what());
    }
  }
};

using namespace ifilt;

extern "C" {

ifilt_status ifilt_server_create(const ifilt_server_opts* opts, ifilt_server* out) {
  try {
    if (!out) fail(IFILT_EINVAL, "null output");
    *out = nullptr;
    auto* s = new ifilt_server_s();
    if (opts) s->opts = *opts;
    if (s->opts.max_lanes < 0 || s->opts.check_every < 0 || s->opts.memory_budget < 0 || s->opts.reserve < 0) {
      delete s;
      fail(IFILT_EINVAL, "negative server option");
    }
    cudaGetDevice(&s->device);
    if (s->opts.memory_budget > 0) {
      s->budget = s->opts.memory_budget;
    } else {
      size_t fr = 0, tot = 0;
      cudaError_t e = cudaMemGetInfo(&fr, &tot);
      if (e != cudaSuccess) {
        delete s;
        fail(IFILT_ECUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
      }
      const int64_t reserve = s->opts.reserve > 0 ? s->opts.reserve : (int64_t)2 << 30;
      s->budget = std::max<int64_t>((int64_t)fr - reserve, 1 << 20);
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return IFILT_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFILT_ENOMEM;
  }
}

ifilt_status ifilt_server_submit(ifilt_server s, ifilt_mesh mesh, const ifilt_solve_opts* o, int32_t n_fields,
                                 const double* fields, int32_t n_k, const double* k, double* out,
                                 ifilt_col_stats* stats, int64_t* request) {
  try {
    if (!s || !mesh || !o || !fields || !k || !out || !request) fail(IFILT_EINVAL, "null argument");
    if (mesh->device < 0) fail(IFILT_EINVAL, "mesh is not uploaded");
    if (n_fields <= 0 || n_k <= 0) fail(IFILT_EINVAL, "n_fields and n_k must be positive");
    if (o->order < 1 || o->order > mesh->host.max_order) fail(IFILT_EINVAL, "order outside the mesh's range");
    if (!(o->tol > 0.0)) fail(IFILT_EINVAL, "tol must be positive");
    if (!(o->err_tol >= 0.0) || !std::isfinite(o->err_tol)) fail(IFILT_EINVAL, "err_tol must be >= 0 and finite");
    if (o->precision < IFILT_PREC_FP64 || o->precision > IFILT_PREC_BF16_IR) fail(IFILT_EINVAL, "unknown precision");
    if (o->precond < IFILT_PRECOND_NONE || o->precond > IFILT_PRECOND_MG) fail(IFILT_EINVAL, "unknown precond");
    if (o->n2_solver < IFILT_N2_AUTO || o->n2_solver > IFILT_N2_COMPLEX) fail(IFILT_EINVAL, "unknown n2_solver");
    if (o->order >= 3 && o->n2_solver == IFILT_N2_COMPLEX)
      fail(IFILT_EINVAL, "the complex factorisation serves order 2 only");
    if (o->mg_cycle != IFILT_MG_V && o->mg_cycle != IFILT_MG_W12) fail(IFILT_EINVAL, "unknown mg_cycle");
    if (o->precond == IFILT_PRECOND_MG &&
        (o->precision == IFILT_PREC_FP64 || !(o->order == 1 || ifilt::complex_form(*o))))
      fail(IFILT_EINVAL, "multigrid preconditioning needs FP32/BF16 and order 1 or the complex n = 2 form");
    for (int32_t j = 0; j < n_k; j++)
      if (!(k[j] > 0.0)) fail(IFILT_EINVAL, "k must be positive");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) fail(IFILT_EINVAL, "server stopped after an error: %s", s->error.c_str());
    if (s->stopping) fail(IFILT_EINVAL, "server is stopping");
    Request r;
    r.id = s->next_id++;
    r.mesh = mesh;
    r.opts = *o;
    r.F = n_fields;
    r.fields = fields;
    r.k.assign(k, k + n_k);
    r.out = out;
    r.stats = stats;
    r.t_submit = s->now();
    *request = r.id;
    s->reqs[r.id] = std::move(r);
    s->incoming.push_back(*request);
    s->cv_work.notify_one();
    return IFILT_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  }
}

ifilt_status ifilt_server_wait(ifilt_server s, int64_t request, int32_t timeout_ms, ifilt_request_info* info) {
  try {
    if (!s || !info) fail(IFILT_EINVAL, "null argument");
    if (timeout_ms < 0) fail(IFILT_EINVAL, "timeout must be >= 0");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request);
    if (it == s->reqs.end()) fail(IFILT_EINVAL, "unknown request %lld", (long long)request);
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return it->second.state >= 2; });
    const Request& r = it->second;
    info->state = r.state;
    info->status = r.status;
    info->columns = r.columns;
    info->columns_done = r.done;
    info->t_submit = r.t_submit;
    info->t_start = r.t_start;
    info->t_done = r.t_done;
    return IFILT_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  }
}

ifilt_status ifilt_server_forget(ifilt_server s, int64_t request) {
  if (!s) return IFILT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end() || it->second.state < 2) {
    set_last_error("unknown or unfinished request");
    return IFILT_EINVAL;
  }
  s->reqs.erase(it);
  return IFILT_OK;
}

double ifilt_server_now(ifilt_server s) { return s ? s->now() : 0.0; }

void ifilt_server_destroy(ifilt_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->engines) {
    kv.second.engine.reset();
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
  delete s;
}

}  // extern "C"
