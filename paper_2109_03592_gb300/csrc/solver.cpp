// Jacobi-preconditioned CG on the device (Sec. 2: "iterative solvers with
// proper preconditioners"; Sec. 3: reductions by hand-written kernels and
// data kept resident on the GPU).
//
// One CG iteration is three kernels:
//   ax  : p <- z + beta p (prologue), w = A_L p, <p, A_L p> -> alpha
//   gs  : w <- mask QQ^T w
//   upd : x += alpha p, r -= alpha w, z = M^{-1} r, <r,z>, <r,r> -> beta, stop test
// All scalars live in a device PcgState, so K iterations are captured once
// into a CUDA graph and replayed; the host reads the state once per chunk
// (double-buffered, so the GPU always has the next chunk queued) and stops
// when the device flags convergence, breakdown or maxit.
//
// Mixed precision (FP64 outer refinement around an FP32 inner PCG): the
// residual r = b - A x is formed in FP64 (FP64 factors), normalised and
// rounded to FP32, solved by the FP32 PCG (FP32 factors, fields and
// M^{-1}; inner products of FP32 products summed in compensated FP32 per
// thread and FP64 across threads), and the FP32 correction is added to x in
// FP64; repeated until the FP64 residual meets the tolerance.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>

#include "kernels.h"
#include "sem_internal.h"
#include "solver.h"

namespace sem {

constexpr int kChunk = 8;  // CG iterations per graph launch

static void destroy_ws(Workspace* ws) {
  if (!ws) return;
  if (ws->s) cudaStreamSynchronize(ws->s);
  for (GraphSlot* g : {&ws->g64, &ws->g32})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  for (void* p : {(void*)ws->x, (void*)ws->r, (void*)ws->z, (void*)ws->p, (void*)ws->w, (void*)ws->minv,
                  (void*)ws->b, (void*)ws->x32, (void*)ws->r32, (void*)ws->z32, (void*)ws->p32, (void*)ws->w32,
                  (void*)ws->minv32, (void*)ws->p32b, (void*)ws->pb, (void*)ws->st, (void*)ws->part_ax, (void*)ws->part_vec})
    if (p) cudaFree(p);
  if (ws->sth) cudaFreeHost(ws->sth);
  for (cudaEvent_t e : {ws->e0, ws->e1, ws->eu, ws->ev[0], ws->ev[1]})
    if (e) cudaEventDestroy(e);
  if (ws->s) cudaStreamDestroy(ws->s);
  delete ws;
}

void free_ws(Workspace* ws) { destroy_ws(ws); }

void release_workspace(sem_mesh* m) {
  std::lock_guard<std::mutex> lk(m->ws_mutex);
  destroy_ws(m->ws);
  m->ws = nullptr;
  for (Workspace* w : m->spare_ws) destroy_ws(w);
  m->spare_ws.clear();
}

static int max_ax_grid(const sem_mesh* m) {
  int epb = 1 << 30;
  for (int v = 0; v < ax_num_variants(); ++v) epb = std::min(epb, ax_elems_per_block(m->N, v));
  return (int)((m->E + epb - 1) / epb);
}

sem_status alloc_ws(sem_mesh* m, Workspace** out) {
  Workspace* ws = new Workspace();
  ws->n = m->n_local;
  const size_t n = (size_t)m->n_local;
  auto fail = [&](cudaError_t e, const char* what) {
    sem_status st = cuda_fail(e, what);
    destroy_ws(ws);
    return st;
  };
  cudaError_t e = cudaSuccess;
  for (double** p : {&ws->x, &ws->r, &ws->z, &ws->p, &ws->w, &ws->minv, &ws->b, &ws->pb})
    if ((e = cudaMalloc((void**)p, n * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc workspace");
  for (float** p : {&ws->x32, &ws->r32, &ws->z32, &ws->p32, &ws->w32, &ws->minv32, &ws->p32b})
    if ((e = cudaMalloc((void**)p, n * sizeof(float))) != cudaSuccess) return fail(e, "cudaMalloc workspace");
  if ((e = cudaMalloc((void**)&ws->st, sizeof(PcgState))) != cudaSuccess) return fail(e, "cudaMalloc state");
  if ((e = cudaMalloc((void**)&ws->part_ax, (size_t)max_ax_grid(m) * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMalloc partials");
  if ((e = cudaMalloc((void**)&ws->part_vec, 3 * (size_t)vec_grid() * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMalloc partials");
  if ((e = cudaMallocHost((void**)&ws->sth, 2 * sizeof(PcgState))) != cudaSuccess) return fail(e, "cudaMallocHost");
  if ((e = cudaStreamCreateWithFlags(&ws->s, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
  for (cudaEvent_t* ev : {&ws->e0, &ws->e1})
    if ((e = cudaEventCreate(ev)) != cudaSuccess) return fail(e, "event");
  for (cudaEvent_t* ev : {&ws->eu, &ws->ev[0], &ws->ev[1]})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  *out = ws;
  return SEM_OK;
}

// ---- local operator dispatch ---------------------------------------------------

cudaError_t ax64(const sem_mesh* m, const double* u, double* w, double h1, double h2, bool fused,
                        const double* z, double* p, PcgState* st, double* part, cudaStream_t s, double* pout) {
  if (m->fp64_df) {
    AxDFParams a{u,      w, m->opG32(), m->opG32lo(), m->opB32(), m->opB32lo(), m->D32, m->D32lo, h1, h2,
                 h2 != 0.0, m->E, z, p, st, part, m->eo64, m->eodf, pout};
    return launch_ax_df(m->N, fused ? m->ax_var_dff : m->ax_var[2], fused, a, s, nullptr);
  }
  AxParams<double> a{u, w, m->opG64(), m->opB64(), m->D64, h1, h2, h2 != 0.0, m->E, z, p, st, part, m->dev_err,
                     pout};
  return launch_ax_f64(m->N, m->ax_var[0], fused, a, s, nullptr);
}

// The native FP64 operator.  The residuals b - A x that decide convergence
// (the outer residuals of the mixed-precision solvers and the final check of
// the FP64 solver) use it: near convergence b - A x cancels to ~1e-10 of the
// terms summed, so the double-float kernel's ~2^-48 rounding, 30x coarser
// than FP64's, would set the attainable residual (measured: the E = 262,144
// pipe stalled above 1e-10 with a 2^-46 input split).
cudaError_t ax64_exact(const sem_mesh* m, const double* u, double* w, double h1, double h2, cudaStream_t s) {
  AxParams<double> a{u, w, m->opG64(), m->opB64(), m->D64, h1, h2, h2 != 0.0, m->E, nullptr, nullptr, nullptr, nullptr,
                     m->dev_err};
  return launch_ax_f64(m->N, m->ax_var[0], false, a, s, nullptr);
}

cudaError_t ax32(const sem_mesh* m, const float* u, float* w, double h1, double h2, bool fused, const float* z,
                 float* p, PcgState* st, double* part, cudaStream_t s, float* pout) {
  AxParams<float> a{u, w, m->opG32(), m->opB32(), m->D32, (float)h1, (float)h2, h2 != 0.0, m->E, z, p, st, part,
                    m->dev_err, pout};
  int var = m->ax_var[1];
  // the bulk-copy kernels read u with 16-byte aligned copies: a caller's
  // unaligned u takes the faster of the register kernels instead
  if (var >= 2 && u && ((uintptr_t)u & 15u)) var = m->ax_ms[1][1] < m->ax_ms[1][0] ? 1 : 0;
  return launch_ax_f32(m->N, var, fused, a, s, nullptr);
}

sem_status apply_local(const sem_mesh* m, const void* u, void* w, double h1, double h2, sem_prec prec,
                       cudaStream_t s) {
  count_launches(1);
  if (prec == SEM_FP64) {
    SEM_CUDA(ax64(m, (const double*)u, (double*)w, h1, h2, false, nullptr, nullptr, nullptr, nullptr, s));
  } else if (prec == SEM_FP32) {
    SEM_CUDA(ax32(m, (const float*)u, (float*)w, h1, h2, false, nullptr, nullptr, nullptr, nullptr, s));
  } else {
    set_error("sem_ax: prec must be SEM_FP64 or SEM_FP32");
    return SEM_ERR_INVALID;
  }
  return SEM_OK;
}

// ---- autotuner -------------------------------------------------------------------

// Times every elements-per-block variant of the FP64, FP32 and double-float
// local operator on this mesh (the mesh's own factors as input) and keeps
// the fastest; FP64 requests use the double-float kernel when it is faster.
// SEM_FP64_KERNEL=native|df forces the FP64 choice.
// Choices are cached per process by (N, log2 E): the first mesh of a shape
// times the variants, later ones reuse its choice, so two meshes of the same
// shape in one process always run the same kernels (and give bitwise-equal
// results).
namespace {
struct TuneKey {
  int N, lg;
  bool operator==(const TuneKey& o) const { return N == o.N && lg == o.lg; }
};
struct TuneVal {
  int var[3];
  int var_dff;
  int df;
  float ms[3][4];
};
std::mutex g_tune_mutex;
std::vector<std::pair<TuneKey, TuneVal>> g_tune;
}  // namespace

static sem_status autotune_measure(sem_mesh* m, cudaStream_t s) {
  const size_t n = (size_t)m->n_local;
  double* w = nullptr;
  SEM_CUDA(cudaMalloc((void**)&w, n * sizeof(double)));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best[3] = {1e30f, 1e30f, 1e30f};
  sem_status status = SEM_OK;
  const int reps = m->E >= 65536 ? 2 : 3;
  for (int kind = 0; kind < 3 && status == SEM_OK; ++kind) {
    if (kind == 2 && !ax_df_available(m->N)) continue;
    for (int v = 0; v < ax_num_variants(); ++v) {
      cudaError_t err = cudaSuccess;
      float total = 0.f;
      for (int rep = 0; rep <= reps && err == cudaSuccess; ++rep) {
        cudaEventRecord(a, s);
        if (kind == 0) {
          AxParams<double> pa{m->B64, w, m->G64, m->B64, m->D64, 1.0, 0.0, 0, m->E, nullptr, nullptr, nullptr, nullptr,
                              m->dev_err};
          err = launch_ax_f64(m->N, v, false, pa, s, nullptr);
        } else if (kind == 1) {
          AxParams<float> pa{m->B32, (float*)w, m->G32, m->B32, m->D32, 1.f, 0.f, 0, m->E,
                             nullptr, nullptr, nullptr, nullptr, m->dev_err};
          err = launch_ax_f32(m->N, v, false, pa, s, nullptr);
        } else {
          AxDFParams pa{m->B64, w, m->G32, m->G32lo, m->B32, m->B32lo, m->D32, m->D32lo, 1.0, 0.0, 0, m->E,
                        nullptr, nullptr, nullptr, nullptr, m->eo64, m->eodf};
          err = launch_ax_df(m->N, v, false, pa, s, nullptr);
        }
        cudaEventRecord(b, s);
        if (err == cudaErrorNotSupported) break;  // no such variant for this (N, precision)
        count_launches(1);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) total += ms;  // first run is a warm-up
      }
      if (err == cudaErrorNotSupported) continue;
      if (err != cudaSuccess) {
        status = cuda_fail(err, "autotune");
        break;
      }
      m->ax_ms[kind][v] = total / reps;
      if (total / reps < best[kind]) {
        best[kind] = total / reps;
        m->ax_var[kind] = v;
      }
    }
  }
  m->fp64_df = ax_df_available(m->N) && best[2] < best[0];
  m->ax_var_dff = m->ax_var[2];
  // The fused double-float form (p = z + beta p, A_L p, <p, A_L p>: the FP64
  // CG's operator) is timed on its own: its fastest variant need not be the
  // plain form's.  z is the mass, beta 0, and the state is cleared before
  // every run, so each run does the same work.
  if (status == SEM_OK && ax_df_available(m->N)) {
    double* p = nullptr;
    double* part = nullptr;
    PcgState* st = nullptr;
    cudaError_t err = cudaMalloc((void**)&p, n * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc((void**)&part, ((size_t)m->E + 1) * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc((void**)&st, sizeof(PcgState));
    if (err == cudaSuccess) err = cudaMemsetAsync(p, 0, n * sizeof(double), s);
    float bestf = 1e30f;
    for (int v = 0; v < ax_num_variants() && err == cudaSuccess; ++v) {
      float total = 0.f;
      cudaError_t e2 = cudaSuccess;
      for (int rep = 0; rep <= reps && e2 == cudaSuccess; ++rep) {
        e2 = cudaMemsetAsync(st, 0, sizeof(PcgState), s);
        if (e2 != cudaSuccess) break;
        cudaEventRecord(a, s);
        AxDFParams pa{nullptr, w, m->G32, m->G32lo, m->B32, m->B32lo, m->D32, m->D32lo, 1.0, 0.0, 0, m->E,
                      m->B64, p,  st,     part,     m->eo64, m->eodf};
        e2 = launch_ax_df(m->N, v, true, pa, s, nullptr);
        cudaEventRecord(b, s);
        if (e2 == cudaErrorNotSupported) break;
        count_launches(2);
        if (e2 == cudaSuccess) e2 = cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) total += ms;
      }
      if (e2 == cudaErrorNotSupported) continue;
      if (e2 != cudaSuccess) {
        err = e2;
        break;
      }
      if (total / reps < bestf) {
        bestf = total / reps;
        m->ax_var_dff = v;
      }
    }
    if (p) cudaFree(p);
    if (part) cudaFree(part);
    if (st) cudaFree(st);
    if (err != cudaSuccess) status = cuda_fail(err, "autotune (fused)");
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(w);
  return status;
}

// Times every elements-per-block variant of the FP64, FP32 and double-float
// local operator on this mesh (the mesh's own factors as input) and keeps
// the fastest; FP64 requests use the double-float kernel when it is faster.
// SEM_FP64_KERNEL=native|df forces the FP64 choice, SEM_FP32_VARIANT=v an
// FP32 variant and SEM_FP64_DF_VARIANT=v a double-float variant (which then
// serves FP64 requests) that exists for this order.
sem_status autotune_mesh(sem_mesh* m, cudaStream_t s) {
  int lg = 0;
  while ((1LL << (lg + 1)) <= m->E) ++lg;
  const TuneKey key{m->N, lg};
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (auto& kv : g_tune)
      if (kv.first == key) {
        for (int k = 0; k < 3; ++k) m->ax_var[k] = kv.second.var[k];
        m->ax_var_dff = kv.second.var_dff;
        m->fp64_df = kv.second.df;
        std::memcpy(m->ax_ms, kv.second.ms, sizeof(m->ax_ms));
        goto forced;
      }
  }
  {
    sem_status st = autotune_measure(m, s);
    if (st != SEM_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    TuneVal v;
    for (int k = 0; k < 3; ++k) v.var[k] = m->ax_var[k];
    v.var_dff = m->ax_var_dff;
    v.df = m->fp64_df;
    std::memcpy(v.ms, m->ax_ms, sizeof(v.ms));
    g_tune.push_back({key, v});
  }
forced:
  if (const char* f = std::getenv("SEM_FP64_KERNEL")) {
    if (!std::strcmp(f, "native")) m->fp64_df = 0;
    if (!std::strcmp(f, "df") && ax_df_available(m->N)) m->fp64_df = 1;
  }
  if (const char* f = std::getenv("SEM_FP32_VARIANT")) {
    const int v = std::atoi(f);
    if (v >= 0 && v < ax_num_variants() && m->ax_ms[1][v] > 0.f) m->ax_var[1] = v;
  }
  if (const char* f = std::getenv("SEM_FP64_DF_VARIANT")) {
    const int v = std::atoi(f);
    if (v >= 0 && v < ax_num_variants() && m->ax_ms[2][v] > 0.f) {
      m->ax_var[2] = v;
      m->ax_var_dff = v;
      m->fp64_df = 1;
    }
  }
  return SEM_OK;
}

// ---- CG chunks ---------------------------------------------------------------------

// Iteration j of a chunk, the directions alternating between p and pb and x
// advanced once per two iterations, as in iter32 below.
static sem_status iter64(sem_mesh* m, Workspace* ws, double h1, double h2, int j) {
  double* src = (j & 1) ? ws->pb : ws->p;
  double* dst = (j & 1) ? ws->p : ws->pb;
  SEM_CUDA(ax64(m, nullptr, ws->w, h1, h2, true, ws->z, src, ws->st, ws->part_ax, ws->s, dst));
  SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, ws->st, ws->s));
  VecParams<double> v{ws->x, ws->r, ws->z, dst, ws->w, ws->minv, ws->b, m->wm, ws->n, ws->st, ws->part_vec, src};
  SEM_CUDA(launch_pcg_update<double>(v, ws->s, false, (j & 1) ? 2 : 1));
  return SEM_OK;
}

// Iteration j of a chunk (kChunk is even).  The directions alternate between
// p32 and p32b: iteration j reads p from one and writes z + beta p to the
// other, so the direction of an even j survives the odd j after it, whose
// update then advances x by both (x += alpha_j p_j + alpha_{j+1} p_{j+1}):
// x is read and written once per two iterations instead of every iteration.
// A chunk starts and ends with the direction in p32 and x current; a pause
// after an even j leaves a pair open, which flush_x32 completes.
static sem_status iter32(sem_mesh* m, Workspace* ws, double h1, double h2, int j) {
  float* src = (j & 1) ? ws->p32b : ws->p32;
  float* dst = (j & 1) ? ws->p32 : ws->p32b;
  SEM_CUDA(ax32(m, nullptr, ws->w32, h1, h2, true, ws->z32, src, ws->st, ws->part_ax, ws->s, dst));
  SEM_CUDA(launch_gs<float>(ws->w32, gs_dev(m), 1, ws->st, ws->s));
  VecParams<float> v{ws->x32, ws->r32, ws->z32, dst,   ws->w32, ws->minv32, ws->r32, m->wm,
                     ws->n,   ws->st,  ws->part_vec, src};
  SEM_CUDA(launch_pcg_update<float>(v, ws->s, false, (j & 1) ? 2 : 1));
  return SEM_OK;
}

// After a run of chunks: complete an open pair of x updates (see iter32 and iter64).
static sem_status flush_x32(Workspace* ws) {
  SEM_CUDA(launch_pcg_xflush<float>(ws->x32, ws->p32, ws->p32b, ws->st, ws->n, ws->s));
  count_launches(1);
  return SEM_OK;
}
static sem_status flush_x64(Workspace* ws) {
  SEM_CUDA(launch_pcg_xflush<double>(ws->x, ws->p, ws->pb, ws->st, ws->n, ws->s));
  count_launches(1);
  return SEM_OK;
}

sem_status put_state(Workspace* ws, double tol, int maxit, int done) {
  PcgState h;
  std::memset(&h, 0, sizeof(h));
  h.tol2 = tol * tol;
  h.maxit = maxit;
  h.done = done;
  ws->sth[0] = h;
  SEM_CUDA(cudaMemcpyAsync(ws->st, &ws->sth[0], sizeof(PcgState), cudaMemcpyHostToDevice, ws->s));
  SEM_CUDA(cudaStreamSynchronize(ws->s));  // the pinned staging slot is reused below
  return SEM_OK;
}

sem_status read_state(Workspace* ws, PcgState& out) {
  SEM_CUDA(cudaMemcpyAsync(&ws->sth[0], ws->st, sizeof(PcgState), cudaMemcpyDeviceToHost, ws->s));
  SEM_CUDA(cudaStreamSynchronize(ws->s));
  out = ws->sth[0];
  return SEM_OK;
}

// Capture kChunk iterations into a graph (once per operator/kernel choice).
static sem_status get_graph(sem_mesh* m, Workspace* ws, bool fp32, double h1, double h2) {
  GraphSlot& g = fp32 ? ws->g32 : ws->g64;
  const int var = fp32 ? m->ax_var[1] : (m->fp64_df ? m->ax_var_dff : m->ax_var[0]);
  const int df = fp32 ? 0 : m->fp64_df;
  if (g.exec && g.h1 == h1 && g.h2 == h2 && g.var == var && g.df == df && g.coef_gen == m->coef_gen) return SEM_OK;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  // One eager pass with done = 1 (every kernel returns at once) so that
  // per-kernel attributes are set outside the capture.
  sem_status st = put_state(ws, 0.0, 0, 1);
  if (st != SEM_OK) return st;
  for (int j = 0; j < 2 && st == SEM_OK; ++j) st = fp32 ? iter32(m, ws, h1, h2, j) : iter64(m, ws, h1, h2, j);
  if (st != SEM_OK) return st;
  count_launches(6);
  SEM_CUDA(cudaStreamSynchronize(ws->s));
  cudaGraph_t graph = nullptr;
  SEM_CUDA(cudaStreamBeginCapture(ws->s, cudaStreamCaptureModeThreadLocal));
  static_assert(kChunk % 2 == 0, "the iterations pair their x updates within a chunk");
  for (int k = 0; k < kChunk && st == SEM_OK; ++k) st = fp32 ? iter32(m, ws, h1, h2, k) : iter64(m, ws, h1, h2, k);
  cudaError_t e = cudaStreamEndCapture(ws->s, &graph);
  if (st != SEM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  g.nodes = (int)nodes;
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  g.h1 = h1;
  g.h2 = h2;
  g.coef_gen = m->coef_gen;
  g.var = var;
  g.df = df;
  return SEM_OK;
}

// Replay the chunk graph until the device reports done.
sem_status run_chunks(Workspace* ws, const GraphSlot& gs, int maxit, PcgState& out) {
  cudaGraphExec_t g = gs.exec;
  const int max_chunks = maxit / kChunk + 3;
  for (int c = 0; c < max_chunks; ++c) {
    SEM_CUDA(cudaGraphLaunch(g, ws->s));
    count_launches(gs.nodes);
    SEM_CUDA(cudaMemcpyAsync(&ws->sth[c & 1], ws->st, sizeof(PcgState), cudaMemcpyDeviceToHost, ws->s));
    SEM_CUDA(cudaEventRecord(ws->ev[c & 1], ws->s));
    if (c > 0) {
      SEM_CUDA(cudaEventSynchronize(ws->ev[(c - 1) & 1]));
      if (ws->sth[(c - 1) & 1].done) {
        SEM_CUDA(cudaEventSynchronize(ws->ev[c & 1]));
        out = ws->sth[c & 1];
        return SEM_OK;
      }
    }
  }
  SEM_CUDA(cudaStreamSynchronize(ws->s));
  out = ws->sth[(max_chunks - 1) & 1];
  if (!out.done) {
    set_error("CG did not report completion within maxit iterations");
    return SEM_ERR_DEVICE_TIMEOUT;
  }
  return SEM_OK;
}

struct SolveOut {
  int iters = 0, outer = 0, status = SEM_OK;
  double rel = 0.0;
};

// Plain FP64 PCG on ws->b with initial guess ws->x.  The CG recurrences
// run with the autotuned (double-float or native) fused operator; when the
// recurrence meets the tolerance, the true residual b - A x is recomputed with
// the native FP64 operator and, if it is still above the tolerance (the
// recurrence drifted), CG restarts from x (at most kMaxRestarts times, within
// maxit iterations in total).  res.rel is that true residual.
static sem_status pcg64(sem_mesh* m, Workspace* ws, const sem_solve_opts& o, int maxit, SolveOut& res) {
  constexpr int kMaxRestarts = 3;
  sem_status st = get_graph(m, ws, false, o.h1, o.h2);
  if (st != SEM_OK) return st;
  res.iters = 0;
  for (int pass = 0;; ++pass) {
    st = put_state(ws, o.tol, maxit - res.iters, 0);
    if (st != SEM_OK) return st;
    SEM_CUDA(ax64_exact(m, ws->x, ws->w, o.h1, o.h2, ws->s));
    SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
    SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, 1, ws->s));
    VecParams<double> v{ws->x, ws->r, ws->z, ws->p, ws->w, ws->minv, ws->b, m->wm, ws->n, ws->st, ws->part_vec};
    SEM_CUDA(launch_pcg_init<double>(v, ws->s));
    count_launches(4);
    PcgState s0;
    st = read_state(ws, s0);
    if (st != SEM_OK) return st;
    if (s0.bb == 0.0) {
      SEM_CUDA(cudaMemsetAsync(ws->x, 0, ws->n * sizeof(double), ws->s));
      res.rel = 0.0;
      res.status = SEM_OK;
      return SEM_OK;
    }
    res.rel = std::sqrt(s0.aux / s0.bb);  // true residual of the current x
    res.outer = pass;
    if (res.rel <= o.tol) {
      res.status = SEM_OK;
      return SEM_OK;
    }
    if (pass > kMaxRestarts || res.iters >= maxit) {
      res.status = SEM_ERR_NOT_CONVERGED;
      return SEM_OK;
    }
    PcgState fin = s0;
    st = run_chunks(ws, ws->g64, maxit - res.iters, fin);
    if (st != SEM_OK) return st;
    st = flush_x64(ws);
    if (st != SEM_OK) return st;
    res.iters += fin.iter;
    if (fin.status != SEM_OK) {  // breakdown, or maxit without meeting the tolerance
      res.rel = std::sqrt(fin.rr / fin.bb);
      res.status = fin.status;
      return SEM_OK;
    }
  }
}

// FP64 refinement around FP32 inner PCG (max_outer = 1 and inner_tol = tol
// gives a plain FP32 PCG).
static sem_status pcg_mixed(sem_mesh* m, Workspace* ws, const sem_solve_opts& o, int maxit, double inner_tol,
                            int max_outer, SolveOut& res) {
  sem_status st = get_graph(m, ws, true, o.h1, o.h2);
  if (st != SEM_OK) return st;
  st = put_state(ws, inner_tol, maxit, 0);  // zero arrival counters before the first reduction
  if (st != SEM_OK) return st;
  for (int outer = 0;; ++outer) {
    SEM_CUDA(ax64_exact(m, ws->x, ws->w, o.h1, o.h2, ws->s));
    SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
    SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, 1, ws->s));
    count_launches(3);
    PcgState s0;
    st = read_state(ws, s0);
    if (st != SEM_OK) return st;
    if (s0.bb == 0.0) {
      SEM_CUDA(cudaMemsetAsync(ws->x, 0, ws->n * sizeof(double), ws->s));
      res.rel = 0.0;
      res.outer = outer;
      return SEM_OK;
    }
    res.rel = std::sqrt(s0.aux / s0.bb);
    res.outer = outer;
    if (res.rel <= o.tol) {
      res.status = SEM_OK;
      return SEM_OK;
    }
    if (outer >= max_outer) {
      res.status = SEM_ERR_NOT_CONVERGED;
      return SEM_OK;
    }
    const double rnorm = std::sqrt(s0.aux);
    launch_scale_to_f32(ws->r32, ws->r, 1.0 / rnorm, ws->n, ws->s);
    launch_zero_f32(ws->x32, ws->n, ws->s);
    SEM_CUDA(cudaGetLastError());
    st = put_state(ws, inner_tol, maxit, 0);
    if (st != SEM_OK) return st;
    VecParams<float> v{ws->x32, ws->r32, ws->z32, ws->p32, ws->w32, ws->minv32, ws->r32, m->wm, ws->n, ws->st,
                       ws->part_vec};
    SEM_CUDA(launch_pcg_init<float>(v, ws->s));
    count_launches(3);
    PcgState fin;
    st = run_chunks(ws, ws->g32, maxit, fin);
    if (st != SEM_OK) return st;
    st = flush_x32(ws);
    if (st != SEM_OK) return st;
    res.iters += fin.iter;
    if (fin.status == SEM_ERR_BREAKDOWN) {
      res.status = SEM_ERR_BREAKDOWN;
      return SEM_OK;
    }
    launch_accumulate(ws->x, ws->x32, rnorm, ws->n, ws->s);
    SEM_CUDA(cudaGetLastError());
    count_launches(1);
  }
}

// Mixed precision with reliable updates: CG recurrences in FP32 on the system
// scaled by 1/||b||; x32 holds the increment since the last update.  The
// update kernel pauses the chunk when the FP32 residual has dropped by delta
// since the last replacement (or meets the tolerance); then x += x32 / s in
// FP64, r = b - A64 x is recomputed in FP64 and replaces the FP32 residual,
// and CG continues with its direction p (beta from the new residual).
static sem_status pcg_mixed_reliable(sem_mesh* m, Workspace* ws, const sem_solve_opts& o, int maxit,
                                     double delta, SolveOut& res) {
  sem_status st = get_graph(m, ws, true, o.h1, o.h2);
  if (st != SEM_OK) return st;
  st = put_state(ws, o.tol, maxit, 0);  // zero arrival counters before the first reduction
  if (st != SEM_OK) return st;
  SEM_CUDA(ax64_exact(m, ws->x, ws->w, o.h1, o.h2, ws->s));
  SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
  SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, 1, ws->s));
  count_launches(3);
  PcgState s0;
  st = read_state(ws, s0);
  if (st != SEM_OK) return st;
  if (s0.bb == 0.0) {
    SEM_CUDA(cudaMemsetAsync(ws->x, 0, ws->n * sizeof(double), ws->s));
    res.rel = 0.0;
    return SEM_OK;
  }
  const double bnorm = std::sqrt(s0.bb), scale = 1.0 / bnorm;
  res.rel = std::sqrt(s0.aux) / bnorm;
  if (res.rel <= o.tol) return SEM_OK;
  // The FP32 residual must undershoot the target (gamma * tol) before a
  // replacement checks the true one; with tol itself a true residual just
  // above tol would trigger a replacement every few steps and stall.
  constexpr double kGamma = 0.2;
  st = put_state(ws, kGamma * o.tol, maxit, 0);
  if (st != SEM_OK) return st;
  launch_scale_to_f32(ws->r32, ws->r, scale, ws->n, ws->s);
  launch_zero_f32(ws->x32, ws->n, ws->s);
  VecParams<float> v{ws->x32, ws->r32, ws->z32, ws->p32, ws->w32, ws->minv32, ws->r32, m->wm, ws->n, ws->st,
                     ws->part_vec};
  SEM_CUDA(launch_pcg_init<float>(v, ws->s));
  launch_set_bb(ws->st, 1.0, delta * delta, ws->s);
  SEM_CUDA(cudaGetLastError());
  count_launches(4);
  for (;;) {
    PcgState fin;
    st = run_chunks(ws, ws->g32, maxit, fin);
    if (st != SEM_OK) return st;
    st = flush_x32(ws);
    if (st != SEM_OK) return st;
    res.iters = fin.iter;
    launch_accumulate(ws->x, ws->x32, bnorm, ws->n, ws->s);
    launch_zero_f32(ws->x32, ws->n, ws->s);
    count_launches(2);
    if (fin.status == SEM_ERR_BREAKDOWN || fin.status == SEM_ERR_NOT_CONVERGED) {
      res.status = fin.status;
      return SEM_OK;
    }
    SEM_CUDA(ax64_exact(m, ws->x, ws->w, o.h1, o.h2, ws->s));
    SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
    SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, 0, ws->s));
    count_launches(3);
    st = read_state(ws, s0);
    if (st != SEM_OK) return st;
    res.outer += 1;
    res.rel = std::sqrt(s0.aux) / bnorm;
    if (res.rel <= o.tol) {
      res.status = SEM_OK;
      return SEM_OK;
    }
    if (res.iters >= maxit) {
      res.status = SEM_ERR_NOT_CONVERGED;
      return SEM_OK;
    }
    launch_scale_to_f32(ws->r32, ws->r, scale, ws->n, ws->s);
    SEM_CUDA(launch_pcg_restart<float>(v, ws->s));
    count_launches(2);
  }
}

// Reliable-update threshold of a single solve: measured on the E = 262,144
// pipe, 0.3 gives 5748 FP32 iterations and 22 FP64 replacements in 11.1 s;
// 0.1: 6161 and 12 in 11.7 s; 0.03: 6297 and 8; 0.01: 6785 and 6; 0.001
// stalls.  (Batched solves default to 0.1: each replacement there costs a
// host round trip per request.)
constexpr double kDefaultDelta = 0.3;

static double tuned_inner_tol(int N) {
  (void)N;
  return 1e-4;
}

static sem_status solve_common(const sem_mesh* cm, const double* b, double* x, bool host_io,
                               const sem_solve_opts* opts, sem_solve_result* result, cudaStream_t user) {
  if (!cm || !b || !x || !opts) {
    set_error("sem_pcg_solve: null argument");
    return SEM_ERR_INVALID;
  }
  sem_mesh* m = const_cast<sem_mesh*>(cm);
  sem_solve_opts o = *opts;
  if (!(o.tol > 0.0)) o.tol = 1e-10;
  const int maxit = o.maxit > 0 ? o.maxit : 20000;
  const int max_outer = o.max_outer > 0 ? o.max_outer : 50;
  const double inner_tol = o.inner_tol > 0.0 ? o.inner_tol : tuned_inner_tol(m->N);
  if (o.prec != SEM_FP64 && o.prec != SEM_FP32 && o.prec != SEM_MIXED) {
    set_error("sem_pcg_solve: bad prec");
    return SEM_ERR_INVALID;
  }
  if (!(o.h1 >= 0.0) || !(o.h2 >= 0.0) || (o.h1 == 0.0 && o.h2 == 0.0)) {
    set_error("sem_pcg_solve: need h1 >= 0, h2 >= 0, not both zero");
    return SEM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(m->ws_mutex);
  if (!m->ws) {
    sem_status st = alloc_ws(m, &m->ws);
    if (st != SEM_OK) return st;
  }
  Workspace* ws = m->ws;
  const size_t bytes = (size_t)ws->n * sizeof(double);
  SEM_CUDA(cudaEventRecord(ws->eu, user));
  SEM_CUDA(cudaStreamWaitEvent(ws->s, ws->eu, 0));
  SEM_CUDA(cudaEventRecord(ws->e0, ws->s));
  const cudaMemcpyKind in = host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  SEM_CUDA(cudaMemcpyAsync(ws->b, b, bytes, in, ws->s));
  SEM_CUDA(cudaMemcpyAsync(ws->x, x, bytes, in, ws->s));
  launch_mask(ws->x, m->wm, ws->n, ws->s);
  count_launches(1);
  if (!(ws->minv_h1 == o.h1 && ws->minv_h2 == o.h2)) {
    launch_minv(ws->minv, ws->minv32, m->opdK(), m->opdB(), m->wm, o.h1, o.h2, ws->n, ws->s);
    count_launches(1);
    ws->minv_h1 = o.h1;
    ws->minv_h2 = o.h2;
  }
  SEM_CUDA(cudaGetLastError());
  SolveOut res;
  sem_status st;
  if (o.prec == SEM_FP64)
    st = pcg64(m, ws, o, maxit, res);
  else if (o.prec == SEM_MIXED && o.refine == 0)
    st = pcg_mixed_reliable(m, ws, o, maxit, o.delta > 0.0 ? o.delta : kDefaultDelta, res);
  else if (o.prec == SEM_MIXED)
    st = pcg_mixed(m, ws, o, maxit, inner_tol, max_outer, res);
  else
    st = pcg_mixed(m, ws, o, maxit, o.tol, 1, res);
  if (st != SEM_OK) {
    ws->minv_h1 = NAN;  // state unknown after a failure
    return st;
  }
  const cudaMemcpyKind outk = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  SEM_CUDA(cudaMemcpyAsync(x, ws->x, bytes, outk, ws->s));
  SEM_CUDA(cudaEventRecord(ws->e1, ws->s));
  SEM_CUDA(cudaStreamSynchronize(ws->s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ws->e0, ws->e1);
  if (result) {
    result->iters = res.iters;
    result->outer_iters = res.outer;
    result->rel_res = res.rel;
    result->ms = ms;
    result->status = res.status;
  }
  return (sem_status)res.status;
}

}  // namespace sem

using namespace sem;

extern "C" {

sem_status sem_pcg_solve(const sem_mesh* m, const double* b_dev, double* x_dev, const sem_solve_opts* opts,
                         sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_pcg_solve");
  return solve_common(m, b_dev, x_dev, false, opts, result, (cudaStream_t)stream);
}

sem_status sem_pcg_solve_host(const sem_mesh* m, const double* b_host, double* x_host, const sem_solve_opts* opts,
                              sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_pcg_solve_host");
  return solve_common(m, b_host, x_host, true, opts, result, (cudaStream_t)stream);
}

}  // extern "C"
