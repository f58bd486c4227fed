// Request server: many Poisson/Helmholtz solves in flight on one GPU.
//
// Requests are queued by sem_server_submit and admitted in arrival order
// (first fit) whenever a slot is idle and the request's estimated device
// footprint fits in what is left of the HBM budget.  Each slot is a worker
// thread with its own CUDA stream; it builds the request's mesh and forms
// b = mask QQ^T (B f).  Then:
//   * mixed-precision requests of an odd order N (the serving form) are
//     handed to the engine thread of that order, which admits them into its
//     running batch (continuous batching): one CUDA graph of batched kernels
//     advances all of that order's requests together, and a request joins or
//     leaves between graph launches;
//   * every other request is solved by the slot itself on its own stream.
// Slots and engines run concurrently, so requests overlap on the device.
// Every request uses only its own buffers and reductions, so its result does
// not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "batch.h"
#include "sem_internal.h"

namespace {

struct Request {
  uint64_t id = 0;
  sem_mesh_desc desc{};
  std::vector<double> xyz;
  std::vector<int64_t> vert;
  std::vector<uint8_t> dface;
  std::vector<double> f;
  sem_solve_opts opts{};
  size_t footprint = 0;
  int64_t n_local = 0;
  std::vector<double> x;
  sem_solve_result res{};
  sem_status status = SEM_OK;
  bool done = false;
  std::string error;
  // batched path: device state kept until the engine finishes the request
  sem_mesh* mesh = nullptr;
  double *f_dev = nullptr, *b_dev = nullptr, *x_dev = nullptr;
  sem::batch::Req breq;
  // host wall-clock marks: submitted, taken by a slot, staged (mesh and b
  // built), solve started (admitted into a batch, or at once), completed
  using Clock = std::chrono::steady_clock;
  Clock::time_point t_submit, t_admit, t_staged, t_solve, t_done;
};

double ms_between(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

int64_t local_points(const sem_mesh_desc& d) {
  const int64_t n = d.N + 1;
  int64_t E = 0;
  if (d.kind == SEM_MESH_BOX) E = (int64_t)d.nx * d.ny * d.nz;
  else if (d.kind == SEM_MESH_PIPE) E = (int64_t)d.nc * (d.nc + 4 * d.nr) * d.nzp;
  else E = d.E;
  return E * n * n * n;
}

// Device bytes one request holds while it runs: mesh arrays (~153 B per
// local point), solver workspace (~80 B), the request's f, b, x (24 B) and the
// set-up scratch (8 B), plus a fixed allowance.
size_t estimate_bytes(const sem_mesh_desc& d) { return (size_t)local_points(d) * 272 + (64u << 20); }

}  // namespace

struct EngineThread {
  int N = 0;
  std::thread th;
  std::deque<std::shared_ptr<Request>> ready;  // built, waiting for a batch slot
  std::vector<std::shared_ptr<Request>> active;
};

struct sem_server {
  sem_server_opts opts{};
  std::vector<std::unique_ptr<EngineThread>> engines;  // one per order, created on demand
  std::condition_variable cv_engine;
  size_t budget = 0, in_use = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<std::thread> workers;
  bool stopping = false;
  bool batch = true;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0;
  int running = 0;
};

namespace {

void free_request_device(Request& q) {
  if (q.f_dev) cudaFree(q.f_dev);
  if (q.b_dev) cudaFree(q.b_dev);
  if (q.x_dev) cudaFree(q.x_dev);
  q.f_dev = q.b_dev = q.x_dev = nullptr;
  if (q.mesh) sem_mesh_destroy(q.mesh);
  q.mesh = nullptr;
}

bool batchable(const Request& q) {
  return q.opts.prec == SEM_MIXED && q.opts.refine == 0 && (q.desc.N % 2) == 1;
}

void complete(sem_server* srv, const std::shared_ptr<Request>& q, sem_status st) {
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    q->t_done = Request::Clock::now();
    q->status = st;
    if (st != SEM_OK && q->error.empty()) q->error = sem_last_error();
    q->done = true;
    srv->in_use -= q->footprint;
    srv->running--;
    srv->completed++;
  }
  srv->cv_done.notify_all();
  srv->cv_work.notify_all();
}

void engine_main(sem_server* srv, EngineThread* et) {
  cudaSetDevice(srv->opts.device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  sem::batch::Engine eng(et->N);
  sem_status init_st = eng.init(s);
  for (;;) {
    std::vector<std::shared_ptr<Request>> incoming;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_engine.wait(lk, [&] { return srv->stopping || !et->ready.empty() || !et->active.empty(); });
      if (srv->stopping && et->ready.empty() && et->active.empty()) break;
      while (!et->ready.empty() && et->active.size() + incoming.size() < 32) {
        incoming.push_back(et->ready.front());
        et->ready.pop_front();
      }
    }
    if (!incoming.empty()) {  // admitted together: their FP64 set-up overlaps on the GPU
      std::vector<sem::batch::Req*> qs;
      for (auto& q : incoming) {
        q->t_solve = Request::Clock::now();
        qs.push_back(&q->breq);
      }
      int taken = 0;
      sem_status st = init_st;
      if (st == SEM_OK) st = eng.add_many(qs.data(), (int)qs.size(), &taken);
      if (st != SEM_OK) {  // the engine is not used again: fail the new requests and those it holds
        eng.abandon();
        for (auto& q : incoming) {
          q->x.clear();
          free_request_device(*q);
          complete(srv, q, st);
        }
        for (auto& q : et->active) {
          free_request_device(*q);
          complete(srv, q, st);
        }
        et->active.clear();
        init_st = st;
        continue;
      }
      for (size_t k = 0; k < incoming.size(); ++k) {
        auto& q = incoming[k];
        if ((int)k >= taken) {
          q->x.clear();
          free_request_device(*q);
          complete(srv, q, SEM_ERR_BUSY);
          continue;
        }
        et->active.push_back(q);
      }
    }
    if (init_st == SEM_OK && !eng.idle()) {
      sem_status st = SEM_OK;
      {
        sem::TraceRange trace("sem_server: batch step");
        st = eng.step();
      }
      if (st != SEM_OK) {  // a CUDA failure: fail every request of this engine
        eng.abandon();
        for (auto& q : et->active) {
          free_request_device(*q);
          complete(srv, q, st);
        }
        et->active.clear();
        init_st = st;
        continue;
      }
    }
    for (size_t k = 0; k < et->active.size();) {
      auto q = et->active[k];
      if (!q->breq.finished) {
        ++k;
        continue;
      }
      q->x.resize(q->n_local);
      cudaMemcpyAsync(q->x.data(), q->x_dev, (size_t)q->n_local * sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      free_request_device(*q);
      complete(srv, q, q->breq.status);
      et->active[k] = et->active.back();
      et->active.pop_back();
    }
  }
  cudaStreamDestroy(s);
}

// Build the mesh and b of a batchable request and hand it to its order's engine.
sem_status stage_for_batch(sem_server* srv, const std::shared_ptr<Request>& q, cudaStream_t s) {
  sem_mesh_desc d = q->desc;
  if (d.kind == SEM_MESH_EXPLICIT) {
    d.xyz = q->xyz.data();
    d.vert = q->vert.data();
    d.dirichlet_face = q->dface.data();
  }
  sem_status st = sem_mesh_create(&d, s, &q->mesh);
  if (st != SEM_OK) return st;
  const size_t bytes = (size_t)q->n_local * sizeof(double);
  cudaError_t e = cudaMalloc((void**)&q->f_dev, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&q->b_dev, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&q->x_dev, bytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q->f_dev, q->f.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->x_dev, 0, bytes, s);
  if (e != cudaSuccess) return sem::cuda_fail(e, "server buffers");
  st = sem_rhs(q->mesh, q->f_dev, q->b_dev, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(cudaStreamSynchronize(s));
  q->breq = sem::batch::Req();
  q->breq.m = q->mesh;
  q->breq.b = q->b_dev;
  q->breq.x = q->x_dev;
  q->breq.o = q->opts;
  if (!(q->breq.o.tol > 0.0)) q->breq.o.tol = 1e-10;
  if (q->breq.o.maxit <= 0) q->breq.o.maxit = 20000;
  if (!(q->breq.o.delta > 0.0)) q->breq.o.delta = 0.1;
  q->breq.out = &q->res;
  q->t_staged = Request::Clock::now();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    EngineThread* et = nullptr;
    for (auto& p : srv->engines)
      if (p->N == q->desc.N) et = p.get();
    if (!et) {
      srv->engines.emplace_back(new EngineThread());
      et = srv->engines.back().get();
      et->N = q->desc.N;
      et->th = std::thread(engine_main, srv, et);
    }
    et->ready.push_back(q);
  }
  srv->cv_engine.notify_all();
  return SEM_OK;
}

sem_status run_request(sem_server* srv, Request& q, cudaStream_t s) {
  (void)srv;
  sem_mesh* m = nullptr;
  sem_mesh_desc d = q.desc;
  if (d.kind == SEM_MESH_EXPLICIT) {
    d.xyz = q.xyz.data();
    d.vert = q.vert.data();
    d.dirichlet_face = q.dface.data();
  }
  sem_status st = sem_mesh_create(&d, s, &m);
  if (st != SEM_OK) return st;
  const size_t bytes = (size_t)q.n_local * sizeof(double);
  double *f = nullptr, *b = nullptr, *x = nullptr;
  cudaError_t e = cudaMalloc((void**)&f, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&x, bytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, q.f.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, bytes, s);
  if (e != cudaSuccess) {
    st = sem::cuda_fail(e, "server buffers");
  } else {
    st = sem_rhs(m, f, b, s);
    if (st == SEM_OK) {
      const cudaError_t e2 = cudaStreamSynchronize(s);
      if (e2 != cudaSuccess) st = sem::cuda_fail(e2, "server rhs");
    }
    q.t_staged = q.t_solve = Request::Clock::now();
    if (st == SEM_OK) st = sem_pcg_solve(m, b, x, &q.opts, &q.res, s);
    if (st == SEM_OK || st == SEM_ERR_NOT_CONVERGED || st == SEM_ERR_BREAKDOWN) {
      q.x.resize(q.n_local);
      e = cudaMemcpyAsync(q.x.data(), x, bytes, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = sem::cuda_fail(e, "server copy-out");
    }
  }
  cudaStreamSynchronize(s);
  if (f) cudaFree(f);
  if (b) cudaFree(b);
  if (x) cudaFree(x);
  sem_mesh_destroy(m);
  return st;
}

void worker_main(sem_server* srv) {
  cudaSetDevice(srv->opts.device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Request> q;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      for (;;) {
        if (srv->stopping) break;
        auto it = std::find_if(srv->queue.begin(), srv->queue.end(), [&](const std::shared_ptr<Request>& r) {
          return srv->in_use + r->footprint <= srv->budget;
        });
        if (it != srv->queue.end()) {
          q = *it;
          q->t_admit = Request::Clock::now();
          srv->queue.erase(it);
          srv->in_use += q->footprint;
          srv->running++;
          break;
        }
        srv->cv_work.wait(lk);
      }
      if (!q) break;
    }
    sem::TraceRange trace(srv->batch && batchable(*q) ? "sem_server: stage a request for its batch"
                                                      : "sem_server: solve a request");
    if (srv->batch && batchable(*q)) {
      sem_status st = stage_for_batch(srv, q, s);
      if (st != SEM_OK) {
        cudaStreamSynchronize(s);
        free_request_device(*q);
        complete(srv, q, st);
      }
      continue;  // the engine thread completes it
    }
    sem_status st = run_request(srv, *q, s);
    complete(srv, q, st);
  }
  cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

sem_status sem_server_create(const sem_server_opts* opts, sem_server** out) {
  if (!opts || !out) {
    sem::set_error("sem_server_create: null argument");
    return SEM_ERR_INVALID;
  }
  *out = nullptr;
  if (cudaSetDevice(opts->device) != cudaSuccess) {
    sem::set_error("sem_server_create: bad device");
    return SEM_ERR_CUDA;
  }
  auto* srv = new sem_server();
  srv->opts = *opts;
  if (srv->opts.max_slots <= 0) srv->opts.max_slots = 8;
  if (srv->opts.max_queue <= 0) srv->opts.max_queue = 4096;
  srv->batch = opts->batch == 0;  // 0 (default): batch the serving form; 1: per-request streams only
  srv->budget = opts->hbm_budget_bytes;
  if (srv->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete srv;
      sem::set_error("sem_server_create: cudaMemGetInfo failed");
      return SEM_ERR_CUDA;
    }
    srv->budget = fr / 10 * 8;
  }
  for (int k = 0; k < srv->opts.max_slots; ++k) srv->workers.emplace_back(worker_main, srv);
  *out = srv;
  return SEM_OK;
}

sem_status sem_server_submit(sem_server* srv, const sem_mesh_desc* desc, const double* f_host,
                             const sem_solve_opts* opts, uint64_t* req_id) {
  if (!srv || !desc || !f_host || !opts || !req_id) {
    sem::set_error("sem_server_submit: null argument");
    return SEM_ERR_INVALID;
  }
  if (desc->N < 1 || desc->N > sem::kMaxN) {
    sem::set_error("sem_server_submit: N must be in [1, 11]");
    return SEM_ERR_INVALID;
  }
  auto q = std::make_shared<Request>();
  q->desc = *desc;
  q->n_local = local_points(*desc);
  if (q->n_local <= 0) {
    sem::set_error("sem_server_submit: empty mesh");
    return SEM_ERR_INVALID;
  }
  q->footprint = estimate_bytes(*desc);
  q->opts = *opts;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (q->footprint > srv->budget) {
      srv->rejected++;
      sem::set_error("sem_server_submit: request exceeds the HBM budget");
      return SEM_ERR_OOM;
    }
    if ((int)srv->queue.size() >= srv->opts.max_queue) {
      srv->rejected++;
      sem::set_error("sem_server_submit: queue full");
      return SEM_ERR_BUSY;
    }
  }
  if (desc->kind == SEM_MESH_EXPLICIT) {
    const int64_t E = desc->E;
    q->xyz.assign(desc->xyz, desc->xyz + q->n_local * 3);
    q->vert.assign(desc->vert, desc->vert + 8 * E);
    q->dface.assign(desc->dirichlet_face, desc->dirichlet_face + 6 * E);
  }
  q->f.assign(f_host, f_host + q->n_local);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    q->t_submit = Request::Clock::now();
    if (srv->stopping) {
      sem::set_error("sem_server_submit: server is stopping");
      return SEM_ERR_INVALID;
    }
    q->id = srv->next_id++;
    srv->reqs[q->id] = q;
    srv->queue.push_back(q);
    srv->submitted++;
    *req_id = q->id;
  }
  srv->cv_work.notify_one();
  return SEM_OK;
}

sem_status sem_server_poll(sem_server* srv, uint64_t req_id, int timeout_ms, double* x_host,
                           sem_solve_result* result) {
  return sem_server_poll_timed(srv, req_id, timeout_ms, x_host, result, nullptr);
}

sem_status sem_server_poll_timed(sem_server* srv, uint64_t req_id, int timeout_ms, double* x_host,
                                 sem_solve_result* result, sem_request_timing* timing) {
  if (!srv) {
    sem::set_error("sem_server_poll: null server");
    return SEM_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) {
    sem::set_error("sem_server_poll: unknown request id");
    return SEM_ERR_NOT_FOUND;
  }
  std::shared_ptr<Request> q = it->second;
  auto ready = [&] { return q->done; };
  if (timeout_ms < 0)
    srv->cv_done.wait(lk, ready);
  else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return SEM_ERR_TIMEOUT;
  if (x_host && !q->x.empty()) std::memcpy(x_host, q->x.data(), q->x.size() * sizeof(double));
  if (result) *result = q->res;
  if (timing) {
    const bool ran = q->t_admit.time_since_epoch().count() != 0;  // not cancelled while queued
    const bool staged = q->t_staged.time_since_epoch().count() != 0;
    const bool solved = q->t_solve.time_since_epoch().count() != 0;
    timing->queue_ms = ran ? ms_between(q->t_submit, q->t_admit) : ms_between(q->t_submit, q->t_done);
    timing->setup_ms = ran && staged ? ms_between(q->t_admit, q->t_staged) : 0.0;
    timing->wait_ms = staged && solved ? ms_between(q->t_staged, q->t_solve) : 0.0;
    timing->solve_ms = solved ? ms_between(q->t_solve, q->t_done) : 0.0;
    timing->total_ms = ms_between(q->t_submit, q->t_done);
  }
  srv->reqs.erase(req_id);
  if (q->status != SEM_OK && !q->error.empty()) sem::set_error(q->error);
  return q->status;
}

sem_status sem_server_cancel(sem_server* srv, uint64_t req_id) {
  if (!srv) return SEM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return SEM_ERR_NOT_FOUND;
  auto qit = std::find(srv->queue.begin(), srv->queue.end(), it->second);
  if (qit == srv->queue.end()) return it->second->done ? SEM_OK : SEM_ERR_BUSY;
  srv->queue.erase(qit);
  it->second->status = SEM_ERR_CANCELLED;
  it->second->done = true;
  it->second->t_done = Request::Clock::now();
  srv->cancelled++;
  srv->cv_done.notify_all();
  return SEM_OK;
}

sem_status sem_server_stats_get(sem_server* srv, sem_server_stats* out) {
  if (!srv || !out) return SEM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->rejected = srv->rejected;
  out->cancelled = srv->cancelled;
  out->queued = (int)srv->queue.size();
  out->running = srv->running;
  out->hbm_in_use = srv->in_use;
  out->hbm_budget = srv->budget;
  return SEM_OK;
}

sem_status sem_server_destroy(sem_server* srv) {
  if (!srv) return SEM_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    for (auto& q : srv->queue) {
      q->status = SEM_ERR_CANCELLED;
      q->done = true;
      q->t_done = Request::Clock::now();
      srv->cancelled++;
    }
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
  for (auto& t : srv->workers) t.join();
  srv->cv_engine.notify_all();
  for (auto& e : srv->engines) e->th.join();  // they finish their requests first
  delete srv;
  return SEM_OK;
}

}  // extern "C"
