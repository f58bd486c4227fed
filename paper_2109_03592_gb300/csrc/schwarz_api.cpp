// The overlapping Schwarz preconditioner of Sec. 2, Eq. 6 on the device, and
// PCG with it (FP64, and FP32 inner CG with FP64 reliable updates).
//
//   M^{-1} r = mask QQ^T (W A~_e^{-1} (W r_e))  +  R_0^T A_0^{-1} R_0 r
//
// Set-up (sem_schwarz_create): the 1D eigenpairs of every element's local
// problem on the host (fdm_tables, each distinct problem once), the coarse
// unknowns (element vertices that are not Dirichlet), the 8 x 8 element
// matrices of A_0 = R_0 A R_0^T on the device (the native FP64 operator
// applied to the masked vertex functions), and A_0 assembled on the host and
// inverted on the device (Gauss-Jordan, SPD) when it has at most
// SEM_SCHWARZ_DENSE_COARSE_MAX unknowns.  Larger coarse problems get a fixed
// symmetric two-level cycle (Chebyshev smoothing, aggregate correction).
//
// One CG iteration with this preconditioner is
//   ax (p = z + beta p, w = A_L p, alpha) | gs (w) | update (x, r, <r,r>, stop)
//   | fdm (r -> z) | gs (z) | coarse restrict | gather | dense A_0^{-1} | prolong (z)
//   | rho (<r, z>, beta)
// all reading the device PcgState, so 8 iterations are captured into one
// CUDA graph as for the Jacobi solver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "schwarz.h"
#include "sem_internal.h"
#include "solver.h"

struct sem_schwarz {
  sem_mesh* m = nullptr;
  double h1 = 1.0, h2 = 0.0;
  uint64_t coef_gen = 0;
  int64_t nd = 0;
  int coarse = 0;  // 1: dense A_0^{-1}; 2: one symmetric two-level cycle on A_0
  bool prec32 = false;  // FP64 solves apply the FP32 preconditioner
  int nc = 0;      // coarse unknowns
  size_t dev_bytes = 0;
  double setup_ms = 0.0;
  // local solves
  int32_t* sidx = nullptr;
  double *S64 = nullptr, *lam64 = nullptr, *wtab64 = nullptr, *ftab64 = nullptr;
  float *S32 = nullptr, *lam32 = nullptr, *wtab32 = nullptr, *ftab32 = nullptr;
  // coarse grid
  int32_t* cidx = nullptr;   // [E][8] coarse unknown of each element vertex (-1: Dirichlet)
  int32_t* cptr = nullptr;   // [nc + 1] CSR over the (element, vertex) slots of each unknown
  int64_t* cslot = nullptr;  // slots 8 e + v, ascending per unknown
  double* rc = nullptr;      // [E][8] element restrictions
  double* g = nullptr;       // [nc]
  double* y = nullptr;       // [nc]
  double* Ainv = nullptr;    // [nc][nc]
  // two-level cycle (coarse = 2): CSR of A_0, 1 / diag, aggregates, dense inverse of A_00
  int32_t *acol = nullptr, *agg = nullptr, *aggptr = nullptr, *aggmem = nullptr;
  double *aval = nullptr, *dinv = nullptr, *A00inv = nullptr, *ga = nullptr, *ya = nullptr, *cwork = nullptr;
  sem::CoarseCycle cyc;
  // solver state
  sem::Workspace* ws = nullptr;
  sem::GraphSlot g64, g32;
  std::mutex mu;
};

namespace sem {
namespace {

// Two-level coarse cycle: Chebyshev degree and range [lambda_max / range,
// lambda_max], aggregates of about agg_size unknowns (at most kAggMax), and
// the number of cycles per coarse solve.  SEM_SCHWARZ_CHEB_DEG,
// SEM_SCHWARZ_CHEB_RANGE, SEM_SCHWARZ_AGG_SIZE and SEM_SCHWARZ_CYCLES
// override the defaults (read when a preconditioner is created).
struct CycleParams {
  int deg = 3;
  double range = 20.0;
  int agg_size = 64;
  int cycles = 1;
};
constexpr int kAggMax = 8192;

// Reliable-update threshold of the mixed Schwarz solve.  Schwarz-PCG reduces
// the residual ~17x faster per iteration than Jacobi, so the Jacobi solver's
// 0.3 replaced the residual every ~16 iterations; measured at E = 262,144
// (mixed, tol 1e-10): 0.3: 329 iterations, 20 replacements, 1.93 s; 0.1: 344,
// 11, 1.82 s; 0.03: 327, 7, 1.66 s; 0.01: 351, 6, 1.75 s.
constexpr double kSchwarzDelta = 0.03;

CycleParams cycle_params() {
  CycleParams p;
  if (const char* v = std::getenv("SEM_SCHWARZ_CHEB_DEG")) p.deg = std::max(1, std::min(kChebMaxDeg, std::atoi(v)));
  if (const char* v = std::getenv("SEM_SCHWARZ_CHEB_RANGE")) p.range = std::max(1.5, std::atof(v));
  if (const char* v = std::getenv("SEM_SCHWARZ_AGG_SIZE")) p.agg_size = std::max(2, std::atoi(v));
  if (const char* v = std::getenv("SEM_SCHWARZ_CYCLES")) p.cycles = std::max(1, std::min(8, std::atoi(v)));
  return p;
}

// Device copy of a host array, on the set-up stream (no legacy-stream copies:
// other threads may be capturing graphs).
template <typename T>
sem_status upload(T** dst, const T* src, size_t count, size_t& bytes, cudaStream_t s) {
  SEM_CUDA(cudaMalloc((void**)dst, std::max<size_t>(count, 1) * sizeof(T)));
  bytes += count * sizeof(T);
  if (count) SEM_CUDA(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  return SEM_OK;
}

void release(sem_schwarz* sw) {
  if (sw->ws) free_ws(sw->ws);
  for (GraphSlot* g : {&sw->g64, &sw->g32})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  for (void* p : {(void*)sw->sidx, (void*)sw->S64, (void*)sw->lam64, (void*)sw->wtab64, (void*)sw->ftab64,
                  (void*)sw->S32, (void*)sw->lam32, (void*)sw->wtab32, (void*)sw->ftab32, (void*)sw->cidx,
                  (void*)sw->cptr, (void*)sw->cslot, (void*)sw->rc, (void*)sw->g, (void*)sw->y, (void*)sw->Ainv,
                  (void*)sw->acol, (void*)sw->agg, (void*)sw->aggptr, (void*)sw->aggmem,
                  (void*)sw->aval, (void*)sw->dinv, (void*)sw->A00inv, (void*)sw->ga, (void*)sw->ya, (void*)sw->cwork})
    if (p) cudaFree(p);
}

#define SW_TRY(expr)                    \
  do {                                  \
    sem_status _s = (expr);             \
    if (_s != SEM_OK) return _s;        \
  } while (0)

// The coarse grid: unknowns, gather lists, element matrices and the dense inverse.
sem_status invert_spd(double* M, int nc, cudaStream_t s) {
  double* f = nullptr;
  int* bad = nullptr;
  SEM_CUDA(cudaMalloc((void**)&f, std::max(nc, 1) * sizeof(double)));
  cudaError_t e = cudaMalloc((void**)&bad, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_gj_inverse(M, nc, f, bad, s);
  count_launches(2 * (uint64_t)nc);
  int bad_h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(f);
  if (bad) cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "coarse-grid inverse");
  if (bad_h) {
    set_error("sem_schwarz_create: a coarse-grid matrix is not positive definite");
    return SEM_ERR_BREAKDOWN;
  }
  return SEM_OK;
}

// Recursive coordinate bisection of the points idx[lo, hi) into `parts`
// groups of near-equal size (split across the longest extent at the
// proportional rank; ties broken by index): agg[idx[q]] = group number.
void rcb(std::vector<int32_t>& idx, int64_t lo, int64_t hi, int parts, int first, const std::vector<double>& pts,
         std::vector<int32_t>& agg) {
  if (parts <= 1 || hi - lo <= 1) {
    for (int64_t q = lo; q < hi; ++q) agg[idx[q]] = first;
    return;
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int64_t q = lo; q < hi; ++q)
    for (int a = 0; a < 3; ++a) {
      mn[a] = std::min(mn[a], pts[3 * (size_t)idx[q] + a]);
      mx[a] = std::max(mx[a], pts[3 * (size_t)idx[q] + a]);
    }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
  const int pl = parts / 2;
  const int64_t mid = lo + (hi - lo) * pl / parts;
  std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int32_t u, int32_t v) {
    const double cu = pts[3 * (size_t)u + ax], cv = pts[3 * (size_t)v + ax];
    return cu < cv || (cu == cv && u < v);
  });
  rcb(idx, lo, mid, pl, first, pts, agg);
  rcb(idx, mid, hi, parts - pl, first + pl, pts, agg);
}

// The two-level cycle for a large A_0: CSR assembly, Jacobi scaling,
// Chebyshev coefficients from a power-iteration estimate of lambda_max(D^{-1}
// A_0), aggregates by coordinate bisection and the dense inverse of P^T A_0 P.
sem_status build_cycle(sem_schwarz* sw, const std::vector<int32_t>& cidx, const std::vector<int32_t>& cnt,
                       const std::vector<int64_t>& slots, const std::vector<double>& Ae_h,
                       const std::vector<double>& pts, cudaStream_t s) {
  const int nc = sw->nc;
  // CSR rows: the slots of each unknown in ascending order, then b ascending (a fixed summation order)
  std::vector<int64_t> ptr(nc + 1, 0);
  std::vector<int32_t> col;
  std::vector<double> val, diag(nc, 0.0);
  col.reserve((size_t)nc * 27);
  val.reserve((size_t)nc * 27);
  std::vector<int32_t> rc_col;
  std::vector<double> rc_val;
  for (int c = 0; c < nc; ++c) {
    rc_col.clear();
    rc_val.clear();
    for (int q = cnt[c]; q < cnt[c + 1]; ++q) {
      const int64_t e = slots[q] / 8;
      const int a = (int)(slots[q] % 8);
      for (int b = 0; b < 8; ++b) {
        const int cb = cidx[8 * e + b];
        if (cb < 0) continue;
        const double v = Ae_h[64 * e + 8 * a + b];
        size_t k = 0;
        while (k < rc_col.size() && rc_col[k] != cb) ++k;
        if (k == rc_col.size()) {
          rc_col.push_back(cb);
          rc_val.push_back(v);
        } else {
          rc_val[k] += v;
        }
      }
    }
    std::vector<size_t> ord(rc_col.size());
    for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
    std::sort(ord.begin(), ord.end(), [&](size_t u, size_t v) { return rc_col[u] < rc_col[v]; });
    for (size_t k : ord) {
      col.push_back(rc_col[k]);
      val.push_back(rc_val[k]);
      if (rc_col[k] == c) diag[c] = rc_val[k];
    }
    ptr[c + 1] = (int64_t)col.size();
  }
  std::vector<double> dinv(nc);
  for (int c = 0; c < nc; ++c) {
    if (!(diag[c] > 0.0)) {
      set_error("sem_schwarz_create: a coarse-grid diagonal entry is not positive");
      return SEM_ERR_BREAKDOWN;
    }
    dinv[c] = 1.0 / diag[c];
  }
  // lambda_max of D^{-1/2} A_0 D^{-1/2} by power iteration (deterministic start)
  std::vector<double> v(nc), w(nc), sq(nc);
  for (int c = 0; c < nc; ++c) {
    sq[c] = std::sqrt(dinv[c]);
    v[c] = 1.0 + 0.5 * std::sin(0.7 * c + 0.3);
  }
  double lam = 0.0;
  for (int it = 0; it < 40; ++it) {
    double nv = 0.0;
    for (int c = 0; c < nc; ++c) nv += v[c] * v[c];
    nv = std::sqrt(nv);
    for (int c = 0; c < nc; ++c) v[c] /= nv;
    double rq = 0.0;
    for (int c = 0; c < nc; ++c) {
      double acc = 0.0;
      for (int64_t q = ptr[c]; q < ptr[c + 1]; ++q) acc += val[q] * sq[col[q]] * v[col[q]];
      w[c] = sq[c] * acc;
      rq += v[c] * w[c];
    }
    lam = rq;
    v.swap(w);
  }
  const CycleParams cp = cycle_params();
  const double lmax = 1.1 * lam, lmin = lmax / cp.range;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  CoarseCycle& cy = sw->cyc;
  cy.deg = cp.deg;
  cy.cycles = cp.cycles;
  cy.cheb_c0 = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 1; k < cy.deg; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    cy.cheb_a[k] = rn * rho;
    cy.cheb_b[k] = 2.0 * rn / delta;
    rho = rn;
  }
  // aggregates
  const int na = std::max(1, std::min(kAggMax, nc / cp.agg_size));
  std::vector<int32_t> idx(nc), agg(nc);
  for (int c = 0; c < nc; ++c) idx[c] = c;
  rcb(idx, 0, nc, na, 0, pts, agg);
  std::vector<int32_t> aptr(na + 1, 0), amem(nc);
  for (int c = 0; c < nc; ++c) aptr[agg[c] + 1]++;
  for (int a = 0; a < na; ++a) aptr[a + 1] += aptr[a];
  {
    std::vector<int32_t> fill(aptr.begin(), aptr.end() - 1);
    for (int c = 0; c < nc; ++c) amem[fill[agg[c]]++] = c;
  }
  std::vector<double> A00((size_t)na * na, 0.0);
  for (int c = 0; c < nc; ++c)
    for (int64_t q = ptr[c]; q < ptr[c + 1]; ++q) A00[(size_t)agg[c] * na + agg[col[q]]] += val[q];
  // ELL form, slot-major: row c's k-th entry at k * nc + c; padding entries are (c, 0)
  int width = 0;
  for (int c = 0; c < nc; ++c) width = std::max<int>(width, (int)(ptr[c + 1] - ptr[c]));
  std::vector<int32_t> ecol((size_t)width * nc);
  std::vector<double> evals((size_t)width * nc, 0.0);
  for (int c = 0; c < nc; ++c)
    for (int k = 0; k < width; ++k) {
      const int64_t q = ptr[c] + k;
      const bool has = q < ptr[c + 1];
      ecol[(size_t)k * nc + c] = has ? col[q] : c;
      evals[(size_t)k * nc + c] = has ? val[q] : 0.0;
    }
  size_t& tb = sw->dev_bytes;
  SW_TRY(upload(&sw->acol, ecol.data(), ecol.size(), tb, s));
  SW_TRY(upload(&sw->aval, evals.data(), evals.size(), tb, s));
  SW_TRY(upload(&sw->dinv, dinv.data(), dinv.size(), tb, s));
  SW_TRY(upload(&sw->agg, agg.data(), agg.size(), tb, s));
  SW_TRY(upload(&sw->aggptr, aptr.data(), aptr.size(), tb, s));
  SW_TRY(upload(&sw->aggmem, amem.data(), amem.size(), tb, s));
  SW_TRY(upload(&sw->A00inv, A00.data(), A00.size(), tb, s));
  SEM_CUDA(cudaMalloc((void**)&sw->ga, na * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&sw->ya, na * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&sw->cwork, 3 * (size_t)nc * sizeof(double)));
  tb += (2 * (size_t)na + 3 * (size_t)nc) * sizeof(double);
  SW_TRY(invert_spd(sw->A00inv, na, s));
  cy.nc = nc;
  cy.na = na;
  cy.width = width;
  cy.col = sw->acol;
  cy.val = sw->aval;
  cy.dinv = sw->dinv;
  cy.agg = sw->agg;
  cy.aptr = sw->aggptr;
  cy.amem = sw->aggmem;
  cy.A00inv = sw->A00inv;
  cy.ga = sw->ga;
  cy.ya = sw->ya;
  cy.work = sw->cwork;
  sw->coarse = 2;
  return SEM_OK;
}

sem_status build_coarse(sem_schwarz* sw, const std::vector<uint8_t>& wm_h, const std::vector<double>& xyz,
                        int dense_max, cudaStream_t s) {
  sem_mesh* m = sw->m;
  const int N = m->N, n = m->n;
  const int64_t E = m->E, n3 = (int64_t)n * n * n, P = m->n_local;
  // element vertices: v = (bi, bj, bk) -> local point (N bi, N bj, N bk)
  std::vector<int64_t> vid(8 * E);
  std::vector<uint8_t> vfree(8 * E);
  for (int64_t e = 0; e < E; ++e)
    for (int v = 0; v < 8; ++v) {
      const int64_t l = e * n3 + N * (v & 1) + n * N * ((v >> 1) & 1) + (int64_t)n * n * N * ((v >> 2) & 1);
      vid[8 * e + v] = m->glo[l];
      vfree[8 * e + v] = (wm_h[l] & 0x80) ? 0 : 1;
    }
  std::vector<int64_t> ids;
  for (int64_t q = 0; q < 8 * E; ++q)
    if (vfree[q]) ids.push_back(vid[q]);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  if (ids.empty() || ids.size() > (size_t)INT32_MAX / 32) {
    sw->coarse = 0;
    sw->nc = (int)std::min<size_t>(ids.size(), (size_t)INT32_MAX);
    return SEM_OK;
  }
  const int nc = (int)ids.size();
  sw->nc = nc;
  std::vector<int32_t> cidx(8 * E, -1), cnt(nc + 1, 0);
  for (int64_t q = 0; q < 8 * E; ++q)
    if (vfree[q]) {
      cidx[q] = (int32_t)(std::lower_bound(ids.begin(), ids.end(), vid[q]) - ids.begin());
      cnt[cidx[q] + 1]++;
    }
  for (int c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
  std::vector<int64_t> slots(cnt[nc]);
  std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t q = 0; q < 8 * E; ++q)
    if (cidx[q] >= 0) slots[fill[cidx[q]]++] = q;  // ascending q per unknown

  // element matrices Ae[e][a][b] = (mask phi_a)^T A_L (mask phi_b) with the native FP64 operator
  double *u = nullptr, *w = nullptr, *Ae = nullptr, *xi_d = nullptr;
  struct Tmp {
    double** p[4];
    ~Tmp() {
      for (double** q : p)
        if (*q) cudaFree(*q);
    }
  } tmp{{&u, &w, &Ae, &xi_d}};
  std::vector<double> xi, wq, D;
  gll(N, xi, wq, D);
  SEM_CUDA(cudaMalloc((void**)&u, P * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&w, P * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&Ae, 64 * E * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&xi_d, n * sizeof(double)));
  SEM_CUDA(cudaMemcpyAsync(xi_d, xi.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  for (int b = 0; b < 8; ++b) {
    SEM_CUDA(launch_fill_phi(u, m->wm, xi_d, n, P, b, s));
    SEM_CUDA(ax64_exact(m, u, w, sw->h1, sw->h2, s));
    SEM_CUDA(launch_elem_coarse(w, m->wm, xi_d, n, E, b, Ae, s));
    count_launches(3);
  }
  std::vector<double> Ae_h(64 * E);
  SEM_CUDA(cudaMemcpyAsync(Ae_h.data(), Ae, 64 * E * sizeof(double), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  size_t& tb = sw->dev_bytes;
  SW_TRY(upload(&sw->cidx, cidx.data(), cidx.size(), tb, s));
  SW_TRY(upload(&sw->cptr, cnt.data(), cnt.size(), tb, s));
  SW_TRY(upload(&sw->cslot, slots.data(), slots.size(), tb, s));
  SEM_CUDA(cudaMalloc((void**)&sw->rc, 8 * E * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&sw->g, nc * sizeof(double)));
  SEM_CUDA(cudaMalloc((void**)&sw->y, nc * sizeof(double)));
  tb += (8 * E + 2 * (size_t)nc) * sizeof(double);
  if (nc > dense_max) {
    // coordinates of each unknown's vertex (its first slot's corner point)
    std::vector<double> pts(3 * (size_t)nc);
    for (int c = 0; c < nc; ++c) {
      const int64_t q = slots[cnt[c]], e = q / 8;
      const int v = (int)(q % 8);
      const int64_t l = N * (v & 1) + n * N * ((v >> 1) & 1) + (int64_t)n * n * N * ((v >> 2) & 1);
      for (int a = 0; a < 3; ++a) pts[3 * (size_t)c + a] = xyz[(size_t)e * 3 * n3 + a * n3 + l];
    }
    return build_cycle(sw, cidx, cnt, slots, Ae_h, pts, s);
  }
  // assembled A_0 (element order, then a, b: a fixed summation order)
  std::vector<double> A0((size_t)nc * nc, 0.0);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 8; ++a) {
      const int ca = cidx[8 * e + a];
      if (ca < 0) continue;
      for (int b = 0; b < 8; ++b) {
        const int cb = cidx[8 * e + b];
        if (cb >= 0) A0[(size_t)ca * nc + cb] += Ae_h[64 * e + 8 * a + b];
      }
    }
  SW_TRY(upload(&sw->Ainv, A0.data(), A0.size(), tb, s));
  SW_TRY(invert_spd(sw->Ainv, nc, s));
  sw->coarse = 1;
  return SEM_OK;
}

// z = M^{-1} r in T (st: the CG state inside a solve, nullptr outside).  With
// rho (inside a CG iteration, coarse term present) the last pass, which adds
// the coarse correction, also forms <r, z> and beta (launch_prolong_rho);
// otherwise the caller forms them.
template <typename T>
sem_status apply_t(const sem_schwarz* sw, const T* r, T* z, PcgState* st, double* partial, bool rho, cudaStream_t s) {
  const sem_mesh* m = sw->m;
  constexpr bool f32 = std::is_same<T, float>::value;
  const T* ft = f32 ? (const T*)sw->ftab32 : (const T*)sw->ftab64;
  FdmParams<T> fp{r,
                  z,
                  m->wm,
                  f32 ? (const T*)sw->wtab32 : (const T*)sw->wtab64,
                  sw->sidx,
                  f32 ? (const T*)sw->S32 : (const T*)sw->S64,
                  f32 ? (const T*)sw->lam32 : (const T*)sw->lam64,
                  (T)sw->h1,
                  (T)sw->h2,
                  m->E,
                  st,
                  ft,
                  sw->coarse ? sw->rc : nullptr};
  SEM_CUDA(launch_fdm<T>(m->N, fp, s));  // local solves, and the coarse restriction R_0 r
  SEM_CUDA(launch_gs<T>(z, gs_dev(m), 1, st, s));
  count_launches(2);
  if (sw->coarse) {
    SEM_CUDA(launch_coarse_gather(sw->rc, sw->cptr, sw->cslot, sw->nc, sw->g, st, s));
    if (sw->coarse == 1) {
      SEM_CUDA(launch_dense_symv(sw->Ainv, sw->g, sw->nc, sw->y, st, s));
      count_launches(1);
    } else {
      SEM_CUDA(launch_vcycle(sw->cyc, sw->g, sw->y, st, s));
      count_launches(vcycle_launches(sw->cyc));
    }
    if (rho) {
      SEM_CUDA(launch_prolong_rho<T>(z, r, m->wm, ft, sw->cidx, sw->y, m->n, m->E, st, partial, s));
    } else {  // the same pass without the product
      SEM_CUDA(launch_prolong_rho<T>(z, r, m->wm, ft, sw->cidx, sw->y, m->n, m->E, const_cast<PcgState*>(st),
                                     nullptr, s));
    }
    count_launches(2);
  }
  return SEM_OK;
}

// One CG iteration with the preconditioner (FP64 or FP32 fields).
// FP32: iteration j of a chunk, the directions alternating between p32 and
// p32b and x advanced once per two iterations, as in the Jacobi solver.
sem_status iter_t(sem_schwarz* sw, bool f32, int j) {
  sem_mesh* m = sw->m;
  Workspace* ws = sw->ws;
  const bool fused_rho = sw->coarse != 0;
  if (f32) {
    float* src = (j & 1) ? ws->p32b : ws->p32;
    float* dst = (j & 1) ? ws->p32 : ws->p32b;
    SEM_CUDA(ax32(m, nullptr, ws->w32, sw->h1, sw->h2, true, ws->z32, src, ws->st, ws->part_ax, ws->s, dst));
    SEM_CUDA(launch_gs<float>(ws->w32, gs_dev(m), 1, ws->st, ws->s));
    VecParams<float> v{ws->x32, ws->r32, ws->z32, dst,          ws->w32, nullptr, ws->r32,
                       m->wm,   ws->n,   ws->st,  ws->part_vec, src};
    SEM_CUDA(launch_pcg_update<float>(v, ws->s, true, (j & 1) ? 2 : 1));
    count_launches(3);
    SW_TRY(apply_t<float>(sw, ws->r32, ws->z32, ws->st, ws->part_vec, fused_rho, ws->s));
    if (!fused_rho) {
      SEM_CUDA((launch_pcg_rho<float, float>(ws->r32, ws->z32, nullptr, 1.0, m->wm, ws->n, ws->st, ws->part_vec, ws->s)));
      count_launches(1);
    }
  } else {
    SEM_CUDA(ax64(m, nullptr, ws->w, sw->h1, sw->h2, true, ws->z, ws->p, ws->st, ws->part_ax, ws->s));
    SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, ws->st, ws->s));
    VecParams<double> v{ws->x, ws->r, ws->z, ws->p, ws->w, nullptr, ws->b, m->wm, ws->n, ws->st, ws->part_vec};
    SEM_CUDA(launch_pcg_update<double>(v, ws->s, true));
    count_launches(3);
    if (sw->prec32) {  // z = M32 float(r), back to FP64 with <r, z> and beta
      launch_scale_to_f32(ws->r32, ws->r, 1.0, ws->n, ws->s);
      SW_TRY(apply_t<float>(sw, ws->r32, ws->z32, ws->st, nullptr, false, ws->s));
      SEM_CUDA((launch_pcg_rho<double, float>(ws->r, ws->z32, ws->z, 1.0, m->wm, ws->n, ws->st, ws->part_vec, ws->s)));
      count_launches(2);
      return SEM_OK;
    }
    SW_TRY(apply_t<double>(sw, ws->r, ws->z, ws->st, ws->part_vec, fused_rho, ws->s));
    if (!fused_rho) {
      SEM_CUDA((launch_pcg_rho<double, double>(ws->r, ws->z, nullptr, 1.0, m->wm, ws->n, ws->st, ws->part_vec, ws->s)));
      count_launches(1);
    }
  }
  return SEM_OK;
}

// z = M r for an FP64 r outside the iteration: the FP64 preconditioner, or the FP32 one.
sem_status apply64(sem_schwarz* sw) {
  Workspace* ws = sw->ws;
  if (!sw->prec32) return apply_t<double>(sw, ws->r, ws->z, nullptr, nullptr, false, ws->s);
  launch_scale_to_f32(ws->r32, ws->r, 1.0, ws->n, ws->s);
  SW_TRY(apply_t<float>(sw, ws->r32, ws->z32, nullptr, nullptr, false, ws->s));
  launch_to_f64(ws->z32, ws->z, ws->n, ws->s);
  count_launches(2);
  SEM_CUDA(cudaGetLastError());
  return SEM_OK;
}

sem_status get_graph(sem_schwarz* sw, bool f32) {
  GraphSlot& g = f32 ? sw->g32 : sw->g64;
  sem_mesh* m = sw->m;
  const int var = f32 ? m->ax_var[1] : (m->fp64_df ? m->ax_var[2] : m->ax_var[0]);
  const int df = f32 ? 0 : m->fp64_df;
  if (g.exec && g.var == var && g.df == df) return SEM_OK;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  Workspace* ws = sw->ws;
  // one eager pass with done = 1 (every kernel returns at once): per-kernel
  // attributes are set outside the capture
  SW_TRY(put_state(ws, 0.0, 0, 1));
  SW_TRY(iter_t(sw, f32, 0));
  if (f32) SW_TRY(iter_t(sw, f32, 1));
  SEM_CUDA(cudaStreamSynchronize(ws->s));
  cudaGraph_t graph = nullptr;
  SEM_CUDA(cudaStreamBeginCapture(ws->s, cudaStreamCaptureModeThreadLocal));
  sem_status st = SEM_OK;
  static_assert(kSolveChunk % 2 == 0, "the FP32 iterations pair their x updates within a chunk");
  for (int k = 0; k < kSolveChunk && st == SEM_OK; ++k) st = iter_t(sw, f32, k);
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
  g.var = var;
  g.df = df;
  return SEM_OK;
}

struct Out {
  int iters = 0, outer = 0, status = SEM_OK;
  double rel = 0.0;
};

// r = b - A x with the native FP64 operator; st->aux = <r, r>, st->bb = <b, b> (set_bb).
sem_status true_residual(sem_schwarz* sw, int set_bb) {
  sem_mesh* m = sw->m;
  Workspace* ws = sw->ws;
  SEM_CUDA(ax64_exact(m, ws->x, ws->w, sw->h1, sw->h2, ws->s));
  SEM_CUDA(launch_gs<double>(ws->w, gs_dev(m), 1, nullptr, ws->s));
  SEM_CUDA(launch_residual(ws->r, ws->b, ws->w, m->wm, ws->n, ws->st, ws->part_vec, set_bb, ws->s));
  count_launches(3);
  return SEM_OK;
}

// FP64 PCG with the FP64 preconditioner; the true residual (native FP64
// operator) is checked once the recurrence meets tol, with restarts as in the
// Jacobi solver.
sem_status pcg64(sem_schwarz* sw, double tol, int maxit, Out& res) {
  constexpr int kMaxRestarts = 3;
  Workspace* ws = sw->ws;
  sem_mesh* m = sw->m;
  SW_TRY(get_graph(sw, false));
  for (int pass = 0;; ++pass) {
    SW_TRY(put_state(ws, tol, maxit - res.iters, 0));
    SW_TRY(true_residual(sw, 1));
    SW_TRY(apply64(sw));
    VecParams<double> v{ws->x, ws->r, ws->z, ws->p, ws->w, nullptr, ws->b, m->wm, ws->n, ws->st, ws->part_vec};
    SEM_CUDA(launch_pcg_init<double>(v, ws->s, true));
    count_launches(1);
    PcgState s0;
    SW_TRY(read_state(ws, s0));
    if (s0.bb == 0.0) {
      SEM_CUDA(cudaMemsetAsync(ws->x, 0, ws->n * sizeof(double), ws->s));
      res.rel = 0.0;
      return SEM_OK;
    }
    res.rel = std::sqrt(s0.aux / s0.bb);
    res.outer = pass;
    if (res.rel <= tol) return SEM_OK;
    if (pass > kMaxRestarts || res.iters >= maxit) {
      res.status = SEM_ERR_NOT_CONVERGED;
      return SEM_OK;
    }
    PcgState fin = s0;
    SW_TRY(run_chunks(ws, sw->g64, maxit - res.iters, fin));
    res.iters += fin.iter;
    if (fin.status != SEM_OK) {
      res.rel = std::sqrt(fin.rr / fin.bb);
      res.status = fin.status;
      return SEM_OK;
    }
  }
}

// FP32 CG (FP32 operator and preconditioner) on the system scaled by 1/||b||,
// with FP64 reliable updates: when the FP32 residual has dropped by delta
// since the last replacement (or below 0.2 tol), x += x32 ||b|| in FP64, the
// true residual is recomputed in FP64 (native operator) and replaces r32, z32
// = M^{-1} r32 is formed again and CG continues with its direction p.
sem_status pcg_mixed(sem_schwarz* sw, double tol, int maxit, double delta, Out& res) {
  Workspace* ws = sw->ws;
  sem_mesh* m = sw->m;
  SW_TRY(get_graph(sw, true));
  SW_TRY(put_state(ws, tol, maxit, 0));
  SW_TRY(true_residual(sw, 1));
  PcgState s0;
  SW_TRY(read_state(ws, s0));
  if (s0.bb == 0.0) {
    SEM_CUDA(cudaMemsetAsync(ws->x, 0, ws->n * sizeof(double), ws->s));
    res.rel = 0.0;
    return SEM_OK;
  }
  const double bnorm = std::sqrt(s0.bb), scale = 1.0 / bnorm;
  res.rel = std::sqrt(s0.aux) / bnorm;
  if (res.rel <= tol) return SEM_OK;
  constexpr double kGamma = 0.2;
  SW_TRY(put_state(ws, kGamma * tol, maxit, 0));
  launch_scale_to_f32(ws->r32, ws->r, scale, ws->n, ws->s);
  launch_zero_f32(ws->x32, ws->n, ws->s);
  count_launches(2);
  SW_TRY(apply_t<float>(sw, ws->r32, ws->z32, nullptr, nullptr, false, ws->s));
  VecParams<float> v{ws->x32, ws->r32, ws->z32, ws->p32, ws->w32, nullptr, ws->r32, m->wm, ws->n, ws->st,
                     ws->part_vec};
  SEM_CUDA(launch_pcg_init<float>(v, ws->s, true));
  launch_set_bb(ws->st, 1.0, delta * delta, ws->s);
  SEM_CUDA(cudaGetLastError());
  count_launches(2);
  for (;;) {
    PcgState fin;
    SW_TRY(run_chunks(ws, sw->g32, maxit, fin));
    SEM_CUDA(launch_pcg_xflush<float>(ws->x32, ws->p32, ws->p32b, ws->st, ws->n, ws->s));  // an open pair of x updates
    count_launches(1);
    res.iters = fin.iter;
    launch_accumulate(ws->x, ws->x32, bnorm, ws->n, ws->s);
    launch_zero_f32(ws->x32, ws->n, ws->s);
    count_launches(2);
    if (fin.status == SEM_ERR_BREAKDOWN || fin.status == SEM_ERR_NOT_CONVERGED) {
      res.status = fin.status;
      return SEM_OK;
    }
    SW_TRY(true_residual(sw, 0));
    SW_TRY(read_state(ws, s0));
    res.outer += 1;
    res.rel = std::sqrt(s0.aux) / bnorm;
    if (res.rel <= tol) return SEM_OK;
    if (res.iters >= maxit) {
      res.status = SEM_ERR_NOT_CONVERGED;
      return SEM_OK;
    }
    launch_scale_to_f32(ws->r32, ws->r, scale, ws->n, ws->s);
    count_launches(1);
    SW_TRY(apply_t<float>(sw, ws->r32, ws->z32, nullptr, nullptr, false, ws->s));
    SEM_CUDA(launch_pcg_restart<float>(v, ws->s, true));
    count_launches(1);
  }
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" {

sem_status sem_schwarz_create(const sem_mesh* mesh, double h1, double h2, int flags, sem_schwarz** out) {
  SEM_TRACE("sem_schwarz_create");
  if (!mesh || !out) {
    set_error("sem_schwarz_create: null argument");
    return SEM_ERR_INVALID;
  }
  *out = nullptr;
  if (!(h1 >= 0.0) || !(h2 >= 0.0) || (h1 == 0.0 && h2 == 0.0) || !std::isfinite(h1) || !std::isfinite(h2)) {
    set_error("sem_schwarz_create: need finite h1 >= 0, h2 >= 0, not both zero");
    return SEM_ERR_INVALID;
  }
  sem_mesh* m = const_cast<sem_mesh*>(mesh);
  if (m->cG64 || m->cB64) {
    set_error("sem_schwarz_create: the separable local solves take scalar h1, h2 (the mesh has per-point "
              "coefficients)");
    return SEM_ERR_INVALID;
  }
  const auto t0 = std::chrono::steady_clock::now();
  SEM_CUDA(cudaSetDevice(m->device));
  sem_schwarz* sw = new sem_schwarz();
  sw->m = m;
  sw->h1 = h1;
  sw->h2 = h2;
  sw->coef_gen = m->coef_gen;
  auto fail = [&](sem_status st) {
    release(sw);
    delete sw;
    return st;
  };
  cudaStream_t s = nullptr;
  {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_fail(e, "stream"));
  }
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } guard{s};
  const int N = m->N, n = N + 1;
  const int64_t E = m->E, P = m->n_local;
  // host copies of the coordinates and the point flags
  std::vector<double> xyz(3 * P);
  std::vector<uint8_t> wm_h(P);
  cudaError_t e = cudaMemcpyAsync(xyz.data(), m->xyz, 3 * P * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(wm_h.data(), m->wm, P, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(cuda_fail(e, "sem_schwarz_create: copies"));
  FdmTables t;
  sem_status st = fdm_tables(E, N, m->glo.data(), xyz.data(), m->dface.data(), t);
  if (st != SEM_OK) return fail(st);
  sw->nd = t.nd;
  std::vector<float> S32(t.S.begin(), t.S.end()), lam32(t.lam.begin(), t.lam.end());
  std::vector<double> wtab(128, 0.0), ftab(2 * n);
  for (int q = 1; q < 128; ++q) wtab[q] = 1.0 / std::sqrt((double)q);
  std::vector<double> xi, w, D;
  gll(N, xi, w, D);
  for (int k = 0; k < n; ++k) {
    ftab[k] = 0.5 * (1.0 - xi[k]);
    ftab[n + k] = 0.5 * (1.0 + xi[k]);
  }
  std::vector<float> wtab32(wtab.begin(), wtab.end()), ftab32(ftab.begin(), ftab.end());
  size_t& tb = sw->dev_bytes;
  if ((st = upload(&sw->sidx, t.sidx.data(), t.sidx.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->S64, t.S.data(), t.S.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->lam64, t.lam.data(), t.lam.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->S32, S32.data(), S32.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->lam32, lam32.data(), lam32.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->wtab64, wtab.data(), wtab.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->wtab32, wtab32.data(), wtab32.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->ftab64, ftab.data(), ftab.size(), tb, s)) != SEM_OK) return fail(st);
  if ((st = upload(&sw->ftab32, ftab32.data(), ftab32.size(), tb, s)) != SEM_OK) return fail(st);
  sw->prec32 = (flags & SEM_SCHWARZ_FP32_PRECOND) != 0;
  if (flags & SEM_SCHWARZ_COARSE) {
    // SEM_SCHWARZ_DENSE_MAX lowers the dense limit (to compare the two coarse forms on one mesh)
    int dense_max = SEM_SCHWARZ_DENSE_COARSE_MAX;
    if (const char* v = std::getenv("SEM_SCHWARZ_DENSE_MAX")) dense_max = std::max(0, std::min(dense_max, std::atoi(v)));
    if ((st = build_coarse(sw, wm_h, xyz, dense_max, s)) != SEM_OK) return fail(st);
  }
  sw->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = sw;
  return SEM_OK;
}

sem_status sem_schwarz_destroy(sem_schwarz* sw) {
  if (!sw) return SEM_OK;
  cudaSetDevice(sw->m->device);
  release(sw);
  delete sw;
  return SEM_OK;
}

sem_status sem_schwarz_info(const sem_schwarz* sw, sem_schwarz_info_t* info) {
  if (!sw || !info) {
    set_error("sem_schwarz_info: null argument");
    return SEM_ERR_INVALID;
  }
  info->n_distinct = sw->nd;
  info->n_coarse = sw->nc;
  info->coarse = sw->coarse;
  info->dev_bytes = sw->dev_bytes;
  info->setup_ms = sw->setup_ms;
  return SEM_OK;
}

sem_status sem_schwarz_apply(const sem_schwarz* sw, const void* r_dev, void* z_dev, sem_prec prec, void* stream) {
  SEM_TRACE("sem_schwarz_apply");
  if (!sw || !r_dev || !z_dev || r_dev == z_dev) {
    set_error("sem_schwarz_apply: null argument, or r and z the same array");
    return SEM_ERR_INVALID;
  }
  if (sw->m->coef_gen != sw->coef_gen) {
    set_error("sem_schwarz_apply: the mesh's coefficients changed since the preconditioner was built");
    return SEM_ERR_INVALID;
  }
  SEM_CUDA(cudaSetDevice(sw->m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SEM_FP64) return apply_t<double>(sw, (const double*)r_dev, (double*)z_dev, nullptr, nullptr, false, s);
  if (prec == SEM_FP32) return apply_t<float>(sw, (const float*)r_dev, (float*)z_dev, nullptr, nullptr, false, s);
  set_error("sem_schwarz_apply: prec must be SEM_FP64 or SEM_FP32");
  return SEM_ERR_INVALID;
}

sem_status sem_schwarz_solve(sem_schwarz* sw, const double* b_dev, double* x_dev, const sem_solve_opts* opts,
                             sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_schwarz_solve");
  if (!sw || !b_dev || !x_dev || !opts) {
    set_error("sem_schwarz_solve: null argument");
    return SEM_ERR_INVALID;
  }
  if (opts->h1 != sw->h1 || opts->h2 != sw->h2) {
    set_error("sem_schwarz_solve: opts h1, h2 must be the preconditioner's");
    return SEM_ERR_INVALID;
  }
  if (opts->prec != SEM_FP64 && opts->prec != SEM_MIXED) {
    set_error("sem_schwarz_solve: prec must be SEM_FP64 or SEM_MIXED");
    return SEM_ERR_INVALID;
  }
  if (sw->m->coef_gen != sw->coef_gen) {
    set_error("sem_schwarz_solve: the mesh's coefficients changed since the preconditioner was built");
    return SEM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(sw->mu);
  sem_mesh* m = sw->m;
  SEM_CUDA(cudaSetDevice(m->device));
  if (!sw->ws) {
    sem_status st = alloc_ws(m, &sw->ws);
    if (st != SEM_OK) return st;
  }
  Workspace* ws = sw->ws;
  const double tol = opts->tol > 0.0 ? opts->tol : 1e-10;
  const int maxit = opts->maxit > 0 ? opts->maxit : 20000;
  const size_t bytes = (size_t)ws->n * sizeof(double);
  cudaStream_t user = (cudaStream_t)stream;
  SEM_CUDA(cudaEventRecord(ws->eu, user));
  SEM_CUDA(cudaStreamWaitEvent(ws->s, ws->eu, 0));
  SEM_CUDA(cudaEventRecord(ws->e0, ws->s));
  SEM_CUDA(cudaMemcpyAsync(ws->b, b_dev, bytes, cudaMemcpyDeviceToDevice, ws->s));
  SEM_CUDA(cudaMemcpyAsync(ws->x, x_dev, bytes, cudaMemcpyDeviceToDevice, ws->s));
  launch_mask(ws->x, m->wm, ws->n, ws->s);
  count_launches(1);
  Out res;
  sem_status st = opts->prec == SEM_FP64
                      ? pcg64(sw, tol, maxit, res)
                      : pcg_mixed(sw, tol, maxit, opts->delta > 0.0 ? opts->delta : kSchwarzDelta, res);
  if (st != SEM_OK) return st;
  SEM_CUDA(cudaMemcpyAsync(x_dev, ws->x, bytes, cudaMemcpyDeviceToDevice, ws->s));
  SEM_CUDA(cudaEventRecord(ws->e1, ws->s));
  SEM_CUDA(cudaEventRecord(ws->eu, ws->s));
  SEM_CUDA(cudaStreamWaitEvent(user, ws->eu, 0));
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

}  // extern "C"
