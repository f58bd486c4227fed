// C ABI of the staggered P_N - P_{N-2} pressure space: the weak divergence D,
// the weak gradient D^T and the consistent Poisson operator E = D B^{-1} D^T
// of Sec. 2, Eq. 5 (pressure on the Gauss-Legendre points of order N-2,
// velocity on the GLL points of order N, Sec. 2).
//
// The GL-point data of a mesh (factors F = rho^3 adj(J) [E][9][m^3], and the
// GLL basis values and derivatives at the GL points) are built on the first
// pressure call on that mesh, on the caller's stream, which that call then
// synchronises.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "sem_internal.h"

namespace sem {
namespace {

// Legendre P_m(x) and P_{m-1}(x) by the three-term recurrence.
void legendre2(int m, double x, double& pm, double& pm1) {
  double p0 = 1.0, p1 = x;
  if (m == 0) {
    pm = 1.0;
    pm1 = 0.0;
    return;
  }
  for (int k = 1; k < m; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pm = p1;
  pm1 = p0;
}

// Gauss-Legendre nodes (roots of P_m, ascending) and weights
// rho = 2 / ((1 - x^2) P_m'(x)^2), by Newton from x = cos(pi (i + 3/4) / (m + 1/2)),
// with (1 - x^2) P_m' = m (P_{m-1} - x P_m).
void gauss_legendre(int m, std::vector<double>& z, std::vector<double>& rho) {
  z.assign(m, 0.0);
  rho.assign(m, 0.0);
  for (int i = 0; i < m; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pm, pm1;
      legendre2(m, x, pm, pm1);
      dp = m * (pm1 - x * pm) / (1.0 - x * x);
      const double dx = pm / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double pm, pm1;
    legendre2(m, x, pm, pm1);
    dp = m * (pm1 - x * pm) / (1.0 - x * x);
    z[i] = x;
    rho[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return z[a] < z[b]; });
  std::vector<double> zs(m), rs(m);
  for (int i = 0; i < m; ++i) {
    zs[i] = z[ord[i]];
    rs[i] = rho[ord[i]];
  }
  z.swap(zs);
  rho.swap(rs);
}

// Ig[i][l] = l_l(z_i) by the barycentric formula on the GLL nodes xi (exactly
// 1 / 0 where z_i is a GLL node), and DIg = Ig D: l_l' has degree N - 1, so it
// equals its own GLL interpolant, l_l'(z) = sum_q l_q(z) D[q][l].
void gl_matrices(int N, std::vector<double>& Ig, std::vector<double>& DIg, std::vector<double>& rho) {
  const int n = N + 1, m = N - 1;
  std::vector<double> xi, w, D, z;
  gll(N, xi, w, D);
  gauss_legendre(m, z, rho);
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (xi[j] - xi[k]);
  Ig.assign(m * n, 0.0);
  for (int i = 0; i < m; ++i) {
    int hit = -1;
    for (int l = 0; l < n; ++l)
      if (z[i] == xi[l]) hit = l;
    if (hit >= 0) {
      Ig[i * n + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int l = 0; l < n; ++l) den += lam[l] / (z[i] - xi[l]);
    for (int l = 0; l < n; ++l) Ig[i * n + l] = (lam[l] / (z[i] - xi[l])) / den;
  }
  DIg.assign(m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < n; ++l) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += Ig[i * n + q] * D[q * n + l];
      DIg[i * n + l] = s;
    }
}

#define SEM_TRY_STATUS(expr)          \
  do {                                \
    sem_status _s = (expr);           \
    if (_s != SEM_OK) return _s;      \
  } while (0)

sem_status check_mesh(const sem_mesh* m, const char* who) {
  if (!m) {
    set_error(std::string(who) + ": null mesh");
    return SEM_ERR_INVALID;
  }
  if (m->N < 2) {
    set_error(std::string(who) + ": the P_N - P_{N-2} pressure space needs N >= 2");
    return SEM_ERR_INVALID;
  }
  return SEM_OK;
}

// Build the mesh's GL-point data once (under its p_mutex).
sem_status ensure_pressure(const sem_mesh* m, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(m->p_mutex);
  if (m->Fgl) return SEM_OK;
  SEM_CUDA(cudaSetDevice(m->device));
  const int N = m->N, n = N + 1, mm = N - 1;
  const int64_t m3 = (int64_t)mm * mm * mm;
  std::vector<double> Ig, DIg, rho;
  gl_matrices(N, Ig, DIg, rho);
  double *F = nullptr, *I_d = nullptr, *DI_d = nullptr, *rho_d = nullptr;
  int* bad_d = nullptr;
  auto release = [&]() {
    if (F) cudaFree(F);
    if (I_d) cudaFree(I_d);
    if (DI_d) cudaFree(DI_d);
    if (rho_d) cudaFree(rho_d);
    if (bad_d) cudaFree(bad_d);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    cudaStreamSynchronize(s);
    release();
    return cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&F, sizeof(double) * 9 * m3 * m->E)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&I_d, sizeof(double) * mm * n)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&DI_d, sizeof(double) * mm * n)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&rho_d, sizeof(double) * mm)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&bad_d, sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMemcpyAsync(I_d, Ig.data(), sizeof(double) * mm * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  if ((e = cudaMemcpyAsync(DI_d, DIg.data(), sizeof(double) * mm * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  if ((e = cudaMemcpyAsync(rho_d, rho.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  if ((e = cudaMemsetAsync(bad_d, 0, sizeof(int), s)) != cudaSuccess) return fail(e, "cudaMemsetAsync");
  if ((e = launch_gl_factors(m->xyz, I_d, DI_d, rho_d, n, mm, m->E, F, bad_d, s)) != cudaSuccess)
    return fail(e, "k_gl_factors");
  count_launches(1);
  int bad = 0;
  if ((e = cudaMemcpyAsync(&bad, bad_d, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  cudaFree(rho_d);
  rho_d = nullptr;
  cudaFree(bad_d);
  bad_d = nullptr;
  if (bad) {
    release();
    set_error("mesh has an element with det(J) <= 0 at a GL point");
    return SEM_ERR_BAD_MESH;
  }
  sem_mesh* mut = const_cast<sem_mesh*>(m);
  mut->dev_bytes += sizeof(double) * (9 * m3 * m->E + 2 * mm * n);
  m->Igl = I_d;
  m->DIgl = DI_d;
  m->Fgl = F;
  return SEM_OK;
}

// FP32 copies of the GL-point data and the reciprocal of the assembled mass,
// for the FP32 operator of the mixed-precision pressure solve (built once,
// under the mesh's p_mutex, after the FP64 data).
sem_status ensure_pressure32(const sem_mesh* m, cudaStream_t s) {
  SEM_TRY_STATUS(ensure_pressure(m, s));
  std::lock_guard<std::mutex> lk(m->p_mutex);
  if (m->Fgl32) return SEM_OK;
  const int N = m->N, n = N + 1, mm = N - 1;
  const int64_t nF = (int64_t)9 * mm * mm * mm * m->E;
  float *F = nullptr, *I = nullptr, *DI = nullptr, *iB = nullptr;
  auto release = [&]() {
    for (float* q : {F, I, DI, iB})
      if (q) cudaFree(q);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    cudaStreamSynchronize(s);
    release();
    return cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&F, sizeof(float) * nF)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&I, sizeof(float) * mm * n)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&DI, sizeof(float) * mm * n)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&iB, sizeof(float) * m->n_local)) != cudaSuccess) return fail(e, "cudaMalloc");
  launch_to_f32(m->Fgl, F, nF, s);
  launch_to_f32(m->Igl, I, (int64_t)mm * n, s);
  launch_to_f32(m->DIgl, DI, (int64_t)mm * n, s);
  launch_recip_f32(m->dB, iB, m->n_local, s);
  count_launches(4);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "pressure FP32 copies");
  sem_mesh* mut = const_cast<sem_mesh*>(m);
  mut->dev_bytes += sizeof(float) * (nF + 2 * mm * n + m->n_local);
  m->Igl32 = I;
  m->DIgl32 = DI;
  m->invB32 = iB;
  m->Fgl32 = F;
  return SEM_OK;
}

// 1 / diag(E), the Jacobi preconditioner of the pressure CG (built once,
// under the mesh's p_mutex, after the FP64 GL-point data).
sem_status ensure_pdiag(const sem_mesh* m, cudaStream_t s) {
  SEM_TRY_STATUS(ensure_pressure(m, s));
  std::lock_guard<std::mutex> lk(m->p_mutex);
  if (m->pdinv) return SEM_OK;
  const int mm = m->N - 1;
  const int64_t np = m->E * mm * mm * mm;
  double* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, sizeof(double) * np);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = launch_pdiag(m->Fgl, m->Igl, m->DIgl, m->wm, m->dB, m->n, mm, m->E, d, 1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    cudaFree(d);
    return cuda_fail(e, "k_pdiag");
  }
  count_launches(1);
  const_cast<sem_mesh*>(m)->dev_bytes += sizeof(double) * np;
  m->pdinv = d;
  return SEM_OK;
}

// q = E p in FP32: weak gradient, masked QQ^T of each component, reciprocal mass, weak divergence.
sem_status apply_E32(const sem_mesh* m, const float* p, float* q, float* work, cudaStream_t s) {
  const int mm = m->N - 1;
  const GsDev g = gs_dev(m);
  SEM_CUDA(launch_pgrad<float>(p, m->Fgl32, m->Igl32, m->DIgl32, m->n, mm, m->E, work, m->n_local, s));
  for (int a = 0; a < 3; ++a) SEM_CUDA(launch_gs<float>(work + a * m->n_local, g, 1, nullptr, s));
  SEM_CUDA(launch_pdiv<float>(work, nullptr, m->invB32, m->Fgl32, m->Igl32, m->DIgl32, m->n, mm, m->E, q, m->n_local,
                              s));
  count_launches(5);
  return SEM_OK;
}

}  // namespace
}  // namespace sem

using namespace sem;

constexpr int kPressureMaxRestarts = 5;
constexpr int kPressureRuGap = 8;  // iterations between residual replacements of the mixed pressure CG

namespace sem {
namespace {

// CG for Eq. 5 on the mean-free pressure space, Pm E Pm p = Pm g with
// Pm = I - 1 1^T / n_p, from p = 0, Jacobi preconditioned (z = Pm(r / diag E))
// or plain.  The iteration runs on the device: its scalars live in a PcgState
// and kChunk iterations are one CUDA graph (E, then k_pcg_psig, k_pcg_pupd and
// k_pcg_pdir), so the host reads the state once per chunk instead of after
// every reduction.  When the recurrence residual meets tol the run pauses and
// the host forms the true residual Pm(g - E p) with the FP64 operator: done if
// it meets tol too; otherwise the FP64 solve restarts from p (at most
// kPressureMaxRestarts times).
// mixed: E applied in FP32 (rounded factors and fields; the FP64 operator is
// bound by GB300's narrow FP64 pipe), FP64 recurrences, and reliable updates:
// the run also pauses when the recurrence residual has dropped by delta since
// the last replacement (at least kPressureRuGap iterations later); the true
// residual then replaces r and CG continues with its direction.  The solve
// stops when the true residual meets tol (the recurrence test is 0.2 tol).
sem_status pressure_cg(const sem_mesh* m, const double* g_dev, double* p_dev, double tol, int maxit, bool mixed,
                       double delta, bool jac, sem_solve_result* result, cudaStream_t us) {
  SEM_TRY_STATUS(ensure_pressure(m, us));
  if (mixed) SEM_TRY_STATUS(ensure_pressure32(m, us));
  if (jac) SEM_TRY_STATUS(ensure_pdiag(m, us));
  // the solve runs on a stream of its own (graph capture needs a non-legacy
  // stream), ordered after the caller's
  cudaStream_t s = nullptr;
  cudaEvent_t ein = nullptr;
  SEM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct Str {
    cudaStream_t* s;
    cudaEvent_t* e;
    ~Str() {
      if (*s) {
        cudaStreamSynchronize(*s);
        cudaStreamDestroy(*s);
      }
      if (*e) cudaEventDestroy(*e);
    }
  } sguard{&s, &ein};
  SEM_CUDA(cudaEventCreateWithFlags(&ein, cudaEventDisableTiming));
  SEM_CUDA(cudaEventRecord(ein, us));
  SEM_CUDA(cudaStreamWaitEvent(s, ein, 0));
  constexpr int kChunk = 8;
  constexpr double kGamma = 0.2;
  const int64_t mm = m->N - 1, np = m->E * mm * mm * mm, nl = m->n_local;
  const int nb = std::max(pressure_red_blocks() + 1, pressure_partials());
  // scratch: r, q, w, z [np]; velocity work [3 n_local]; partials; one sum; the state
  double* buf = nullptr;
  float* buf32 = nullptr;
  PcgState* sth = nullptr;
  const size_t count = 4 * (size_t)np + 3 * (size_t)nl + nb + 1 + (sizeof(PcgState) + 7) / 8;
  SEM_CUDA(cudaMalloc((void**)&buf, count * sizeof(double)));
  cudaGraphExec_t exec = nullptr;
  struct Free {
    double* b;
    float** f;
    PcgState** h;
    cudaGraphExec_t* x;
    ~Free() {
      if (*x) cudaGraphExecDestroy(*x);
      cudaFree(b);
      if (*f) cudaFree(*f);
      if (*h) cudaFreeHost(*h);
    }
  } guard{buf, &buf32, &sth, &exec};
  if (mixed) SEM_CUDA(cudaMalloc((void**)&buf32, (2 * (size_t)np + 3 * (size_t)nl) * sizeof(float)));
  SEM_CUDA(cudaMallocHost((void**)&sth, sizeof(PcgState)));
  double* r = buf;
  double* q = r + np;
  double* w = q + np;
  double* z = w + np;
  double* work = z + np;
  double* partial = work + 3 * nl;
  double* sum_d = partial + nb;
  PcgState* st = reinterpret_cast<PcgState*>(sum_d + 1);
  float* q32 = buf32;
  float* w32 = mixed ? q32 + np : nullptr;
  float* work32 = mixed ? w32 + np : nullptr;
  const GsDev g = gs_dev(m);
  auto read = [&](double& v) -> sem_status {
    SEM_CUDA(cudaMemcpyAsync(&v, sum_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
  };
  auto put = [&]() -> sem_status {
    SEM_CUDA(cudaMemcpyAsync(st, sth, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
  };
  auto get = [&]() -> sem_status {
    SEM_CUDA(cudaMemcpyAsync(sth, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
  };
  uint64_t launches = 0;
  // out = E v in FP64: weak gradient, QQ^T with mask on each component, inverse mass, weak divergence
  auto apply_E = [&](const double* v, double* out) -> sem_status {
    SEM_CUDA(launch_pgrad<double>(v, m->Fgl, m->Igl, m->DIgl, m->n, (int)mm, m->E, work, nl, s));
    for (int a = 0; a < 3; ++a) SEM_CUDA(launch_gs<double>(work + a * nl, g, 1, nullptr, s));
    SEM_CUDA(launch_pdiv<double>(work, m->dB, nullptr, m->Fgl, m->Igl, m->DIgl, m->n, (int)mm, m->E, out, nl, s));
    launches += 5;
    return SEM_OK;
  };
  // z = Pm (dinv r) in place and <r, z>, host-synchronous (start and after replacements)
  auto precondition = [&](double& rz) -> sem_status {
    double zs = 0.0;
    SEM_CUDA(launch_pscale(r, m->pdinv, z, np, partial, sum_d, s));
    SEM_TRY_STATUS(read(zs));
    SEM_CUDA(launch_pshift_dot(z, r, zs / (double)np, np, partial, sum_d, s));
    SEM_TRY_STATUS(read(rz));
    launches += 4;
    return SEM_OK;
  };
  const double* zdir = jac ? z : r;

  cudaEvent_t e0, e1;
  SEM_CUDA(cudaEventCreate(&e0));
  SEM_CUDA(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evguard{e0, e1};
  SEM_CUDA(cudaEventRecord(e0, s));
  // mean of g, then r = q = g - mean, x = 0, <r, r>
  double gsum = 0.0, rr0 = 0.0;
  SEM_CUDA(launch_pdot(g_dev, nullptr, np, partial, sum_d, s));
  SEM_TRY_STATUS(read(gsum));
  SEM_CUDA(launch_pstart(g_dev, gsum / (double)np, r, q, p_dev, np, partial, sum_d, s));
  SEM_TRY_STATUS(read(rr0));
  launches += 4;
  const double gnorm = std::sqrt(rr0);
  int status = SEM_OK, outer = 0, restarts = 0, iters = 0;
  double rel = 0.0;
  if (gnorm > 0.0) {
    double rho = rr0;
    if (jac) {
      SEM_TRY_STATUS(precondition(rho));
      SEM_CUDA(launch_pdir(q, z, 0.0, np, s));
      launches += 1;
    }
    std::memset(sth, 0, sizeof(PcgState));
    sth->rho = rho;
    sth->rr = rr0;
    sth->rr_max = rr0;
    sth->bb = rr0;
    sth->tol2 = tol * tol;
    sth->delta2 = mixed ? delta * delta : 0.0;
    sth->maxit = maxit;
    SEM_TRY_STATUS(put());
    // one iteration, kChunk times in a graph
    auto iteration = [&]() -> sem_status {
      if (mixed) {
        launch_to_f32(q, q32, np, s);
        SEM_TRY_STATUS(apply_E32(m, q32, w32, work32, s));
        launch_to_f64(w32, w, np, s);
      } else {
        SEM_TRY_STATUS(apply_E(q, w));
      }
      SEM_CUDA(launch_pcg_psig(q, w, np, st, partial, s));
      SEM_CUDA(launch_pcg_pupd(jac, mixed, p_dev, r, q, w, m->pdinv, z, np, st, partial, kGamma * kGamma,
                               kPressureRuGap, s));
      SEM_CUDA(launch_pcg_pdir(q, zdir, np, st, s));
      return SEM_OK;
    };
    const int per_iter = mixed ? 10 : 8;
    {
      cudaGraph_t graph = nullptr;
      SEM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      sem_status cst = SEM_OK;
      for (int k = 0; k < kChunk && cst == SEM_OK; ++k) cst = iteration();
      cudaError_t ce = cudaStreamEndCapture(s, &graph);
      if (cst != SEM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return cst;
      }
      SEM_CUDA(ce);
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      SEM_CUDA(ce);
    }
    status = SEM_ERR_NOT_CONVERGED;
    rel = 1.0;
    for (;;) {
      SEM_CUDA(cudaGraphLaunch(exec, s));
      launches += (uint64_t)kChunk * per_iter;
      SEM_TRY_STATUS(get());
      if (!sth->done) continue;
      iters = sth->iter;
      rel = std::sqrt(sth->rr) / gnorm;
      if (!sth->ru) {  // breakdown or the iteration cap
        status = sth->status;
        break;
      }
      // the true residual Pm (g - E x) with the FP64 operator
      double xs = 0.0, rr_t = 0.0;
      SEM_TRY_STATUS(apply_E(p_dev, w));
      SEM_CUDA(launch_pdot(w, nullptr, np, partial, sum_d, s));
      SEM_TRY_STATUS(read(xs));
      SEM_CUDA(launch_presidual_keep(g_dev, gsum / (double)np, w, xs / (double)np, r, np, partial, sum_d, s));
      SEM_TRY_STATUS(read(rr_t));
      launches += 4;
      rel = std::sqrt(rr_t) / gnorm;
      if (std::sqrt(rr_t) <= tol * gnorm) {
        status = SEM_OK;
        break;
      }
      if (sth->iter >= maxit) break;
      double rho_new = rr_t;
      if (jac) SEM_TRY_STATUS(precondition(rho_new));
      if (mixed) {  // replacement: CG keeps its direction
        ++outer;
        SEM_CUDA(launch_pdir(q, zdir, rho_new / sth->rho, np, s));
        sth->rr_max = rr_t;
        sth->last = sth->iter;
      } else {  // restart from x with the true residual
        if (restarts == kPressureMaxRestarts) break;
        ++restarts;
        SEM_CUDA(launch_pdir(q, zdir, 0.0, np, s));
      }
      launches += 1;
      sth->rho = rho_new;
      sth->rr = rr_t;
      sth->done = 0;
      sth->ru = 0;
      sth->status = 0;
      SEM_TRY_STATUS(put());
    }
  }
  SEM_CUDA(cudaEventRecord(e1, s));
  SEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  SEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  count_launches(launches);
  result->iters = iters;
  result->outer_iters = outer;
  result->rel_res = rel;
  result->ms = ms;
  result->status = status;
  return (sem_status)status;
}

}  // namespace
}  // namespace sem

extern "C" {

sem_status sem_pressure_basis(int N, double* zeta_host, double* rho_host, double* Ig_host, double* DIg_host) {
  if (N < 2 || N > kMaxN) {
    set_error("sem_pressure_basis: N must be in [2, 11]");
    return SEM_ERR_INVALID;
  }
  std::vector<double> Ig, DIg, rho, z, r2;
  gl_matrices(N, Ig, DIg, rho);
  gauss_legendre(N - 1, z, r2);
  if (zeta_host) std::copy(z.begin(), z.end(), zeta_host);
  if (rho_host) std::copy(rho.begin(), rho.end(), rho_host);
  if (Ig_host) std::copy(Ig.begin(), Ig.end(), Ig_host);
  if (DIg_host) std::copy(DIg.begin(), DIg.end(), DIg_host);
  return SEM_OK;
}

sem_status sem_pressure_info(const sem_mesh* m, int64_t* n_pressure) {
  sem_status st = check_mesh(m, "sem_pressure_info");
  if (st != SEM_OK) return st;
  if (!n_pressure) {
    set_error("sem_pressure_info: null argument");
    return SEM_ERR_INVALID;
  }
  const int64_t mm = m->N - 1;
  *n_pressure = m->E * mm * mm * mm;
  return SEM_OK;
}

sem_status sem_pressure_factors(const sem_mesh* m, double* F_dev, void* stream) {
  sem_status st = check_mesh(m, "sem_pressure_factors");
  if (st != SEM_OK) return st;
  if (!F_dev) {
    set_error("sem_pressure_factors: null argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure(m, s);
  if (st != SEM_OK) return st;
  const int64_t mm = m->N - 1;
  SEM_CUDA(cudaMemcpyAsync(F_dev, m->Fgl, sizeof(double) * 9 * mm * mm * mm * m->E, cudaMemcpyDeviceToDevice, s));
  return SEM_OK;
}

sem_status sem_pressure_grad(const sem_mesh* m, const double* p_dev, double* u_dev, void* stream) {
  sem_status st = check_mesh(m, "sem_pressure_grad");
  if (st != SEM_OK) return st;
  if (!p_dev || !u_dev) {
    set_error("sem_pressure_grad: null argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure(m, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(launch_pgrad<double>(p_dev, m->Fgl, m->Igl, m->DIgl, m->n, m->N - 1, m->E, u_dev, m->n_local, s));
  count_launches(1);
  return SEM_OK;
}

sem_status sem_pressure_div(const sem_mesh* m, const double* u_dev, double* q_dev, void* stream) {
  sem_status st = check_mesh(m, "sem_pressure_div");
  if (st != SEM_OK) return st;
  if (!u_dev || !q_dev) {
    set_error("sem_pressure_div: null argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure(m, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(launch_pdiv<double>(u_dev, nullptr, nullptr, m->Fgl, m->Igl, m->DIgl, m->n, m->N - 1, m->E, q_dev, m->n_local, s));
  count_launches(1);
  return SEM_OK;
}

sem_status sem_pressure_apply(const sem_mesh* m, const double* p_dev, double* q_dev, double* work_dev, void* stream) {
  SEM_TRACE("sem_pressure_apply");
  sem_status st = check_mesh(m, "sem_pressure_apply");
  if (st != SEM_OK) return st;
  if (!p_dev || !q_dev || !work_dev) {
    set_error("sem_pressure_apply: null argument");
    return SEM_ERR_INVALID;
  }
  const int64_t mm = m->N - 1, np = m->E * mm * mm * mm;
  const double* w0 = work_dev;
  const double* w1 = work_dev + 3 * m->n_local;
  auto overlaps = [&](const double* a) { return a + np > w0 && a < w1; };
  if (overlaps(p_dev) || overlaps(q_dev)) {
    set_error("sem_pressure_apply: work must not overlap p or q");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure(m, s);
  if (st != SEM_OK) return st;
  const GsDev g = gs_dev(m);
  SEM_CUDA(launch_pgrad<double>(p_dev, m->Fgl, m->Igl, m->DIgl, m->n, m->N - 1, m->E, work_dev, m->n_local, s));
  for (int a = 0; a < 3; ++a) SEM_CUDA(launch_gs<double>(work_dev + a * m->n_local, g, 1, nullptr, s));
  SEM_CUDA(launch_pdiv<double>(work_dev, m->dB, nullptr, m->Fgl, m->Igl, m->DIgl, m->n, m->N - 1, m->E, q_dev, m->n_local, s));
  count_launches(5);
  return SEM_OK;
}

sem_status sem_pressure_apply_f32(const sem_mesh* m, const float* p_dev, float* q_dev, float* work_dev, void* stream) {
  SEM_TRACE("sem_pressure_apply_f32");
  sem_status st = check_mesh(m, "sem_pressure_apply_f32");
  if (st != SEM_OK) return st;
  if (!p_dev || !q_dev || !work_dev || p_dev == q_dev) {
    set_error("sem_pressure_apply_f32: null or overlapping argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure32(m, s);
  if (st != SEM_OK) return st;
  return apply_E32(m, p_dev, q_dev, work_dev, s);
}

sem_status sem_pressure_diag(const sem_mesh* m, double* d_dev, void* stream) {
  SEM_TRACE("sem_pressure_diag");
  sem_status st = check_mesh(m, "sem_pressure_diag");
  if (st != SEM_OK) return st;
  if (!d_dev) {
    set_error("sem_pressure_diag: null output");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_pressure(m, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(launch_pdiag(m->Fgl, m->Igl, m->DIgl, m->wm, m->dB, m->n, m->N - 1, m->E, d_dev, 0, s));
  count_launches(1);
  return SEM_OK;
}

sem_status sem_pressure_solve(const sem_mesh* m, const double* g_dev, double* p_dev, const sem_solve_opts* opts,
                              sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_pressure_solve");
  sem_status st = check_mesh(m, "sem_pressure_solve");
  if (st != SEM_OK) return st;
  if (!g_dev || !p_dev || !opts || !result || g_dev == p_dev) {
    set_error("sem_pressure_solve: null or overlapping argument");
    return SEM_ERR_INVALID;
  }
  const double tol = opts->tol > 0 ? opts->tol : 1e-10;
  const int maxit = opts->maxit > 0 ? opts->maxit : 20000;
  *result = sem_solve_result{0, 0, 0.0, 0.0, SEM_OK};
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->precond != SEM_PRECOND_DEFAULT && opts->precond != SEM_PRECOND_NONE &&
      opts->precond != SEM_PRECOND_JACOBI) {
    set_error("sem_pressure_solve: precond must be SEM_PRECOND_DEFAULT, _NONE or _JACOBI");
    return SEM_ERR_INVALID;
  }
  const bool jac = opts->precond != SEM_PRECOND_NONE;
  if (opts->prec != SEM_FP64 && opts->prec != SEM_MIXED) {
    set_error("sem_pressure_solve: prec must be SEM_FP64 or SEM_MIXED");
    return SEM_ERR_INVALID;
  }
  SEM_CUDA(cudaSetDevice(m->device));
  return pressure_cg(m, g_dev, p_dev, tol, maxit, opts->prec == SEM_MIXED, opts->delta > 0.0 ? opts->delta : 0.1, jac,
                     result, s);
}

}  // extern "C"

