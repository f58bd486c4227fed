// C ABI: mesh construction and the operator entry points (sem_ax, sem_gs,
// sem_rhs, sem_apply, sem_jacobi).  The solver lives in solver.cpp and the
// server in server.cpp.
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "kernels.h"
#include "sem_internal.h"
#include "solver.h"

namespace sem {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

sem_status cuda_fail(cudaError_t err, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")");
  return err == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA;
}

namespace {

template <typename T>
sem_status dev_alloc(T** p, size_t count, size_t& tally) {
  *p = nullptr;
  if (count == 0) return SEM_OK;
  cudaError_t err = cudaMalloc((void**)p, count * sizeof(T));
  if (err != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(err, "cudaMalloc");
  }
  tally += count * sizeof(T);
  return SEM_OK;
}

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void free_mesh_arrays(sem_mesh* m) {
  dev_free(m->xyz);
  dev_free(m->G64);
  dev_free(m->B64);
  dev_free(m->G32);
  dev_free(m->G32lo);
  dev_free(m->B32);
  dev_free(m->B32lo);
  dev_free(m->dK);
  dev_free(m->dB);
  dev_free(m->wm);
  dev_free(m->gs_idx);
  dev_free(m->gs_ptr);
  dev_free(m->gs_units);
  dev_free(m->D64);
  dev_free(m->dev_err);
  dev_free(m->D32);
  dev_free(m->D32lo);
  dev_free(m->eo64);
  dev_free(m->eodf);
  dev_free(m->cG64);
  dev_free(m->cG32);
  dev_free(m->cG32lo);
  dev_free(m->cdK);
  dev_free(m->cB64);
  dev_free(m->cB32);
  dev_free(m->cB32lo);
  dev_free(m->cdB);
  dev_free(m->Fgl);
  dev_free(m->pdinv);
  dev_free(m->Igl);
  dev_free(m->DIgl);
  dev_free(m->Fgl32);
  dev_free(m->Igl32);
  dev_free(m->DIgl32);
  dev_free(m->invB32);
}

#define SEM_TRY(expr)                   \
  do {                                  \
    sem_status _s = (expr);             \
    if (_s != SEM_OK) return _s;        \
  } while (0)

// The operator arrays for per-point coefficients, built aside and installed
// only once the coefficients were found valid.
struct CoefArrays {
  double* G64 = nullptr;
  float* G32 = nullptr;
  float* G32lo = nullptr;
  double* dK = nullptr;
  double* B64 = nullptr;
  float* B32 = nullptr;
  float* B32lo = nullptr;
  double* dB = nullptr;
  size_t bytes = 0;
  void release() {
    dev_free(G64);
    dev_free(G32);
    dev_free(G32lo);
    dev_free(dK);
    dev_free(B64);
    dev_free(B32);
    dev_free(B32lo);
    dev_free(dB);
    bytes = 0;
  }
};

size_t coef_bytes(const sem_mesh* m) {
  const size_t P = (size_t)m->n_local;
  return (m->cG64 ? P * (6 * 8 + 6 * 4 + 6 * 4 + 8) : 0) + (m->cB64 ? P * (8 + 4 + 4 + 8) : 0);
}

sem_status build_coef(const sem_mesh* m, const double* h1, const double* h2, CoefArrays& c, cudaStream_t s) {
  const int64_t P = m->n_local;
  const int n = m->n;
  if (h1) {
    SEM_TRY(dev_alloc(&c.G64, 6 * P, c.bytes));
    SEM_TRY(dev_alloc(&c.G32, 6 * P, c.bytes));
    SEM_TRY(dev_alloc(&c.G32lo, 6 * P, c.bytes));
    SEM_TRY(dev_alloc(&c.dK, P, c.bytes));
  }
  if (h2) {
    SEM_TRY(dev_alloc(&c.B64, P, c.bytes));
    SEM_TRY(dev_alloc(&c.B32, P, c.bytes));
    SEM_TRY(dev_alloc(&c.B32lo, P, c.bytes));
    SEM_TRY(dev_alloc(&c.dB, P, c.bytes));
  }
  size_t tmp = 0;
  int* bad_d = nullptr;
  SEM_TRY(dev_alloc(&bad_d, 1, tmp));
  std::unique_ptr<int, void (*)(int*)> bad_guard(bad_d, [](int* p) { cudaFree(p); });
  SEM_CUDA(cudaMemsetAsync(bad_d, 0, sizeof(int), s));
  launch_fold_coef(m->G64, m->B64, h1, h2, c.G64, c.B64, n, P, bad_d, s);
  if (h1) {
    launch_local_diag(c.G64, c.dK, m->D64, n, m->E, s);
    SEM_CUDA(launch_gs<double>(c.dK, gs_dev(m), 0, nullptr, s));
    launch_split_f64(c.G64, c.G32, c.G32lo, 6 * P, s);
  }
  if (h2) {
    SEM_CUDA(cudaMemcpyAsync(c.dB, c.B64, P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SEM_CUDA(launch_gs<double>(c.dB, gs_dev(m), 0, nullptr, s));
    launch_split_f64(c.B64, c.B32, c.B32lo, P, s);
  }
  SEM_CUDA(cudaGetLastError());
  count_launches(1 + (h1 ? 3 : 0) + (h2 ? 2 : 0));
  int bad = 0;
  SEM_CUDA(cudaMemcpyAsync(&bad, bad_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    set_error((bad & 1) ? "sem_mesh_set_coefficients: need finite h1 > 0 at every point"
                        : "sem_mesh_set_coefficients: need finite h2 >= 0 at every point");
    return SEM_ERR_INVALID;
  }
  return SEM_OK;
}

sem_status build_mesh(const sem_mesh_desc& d, cudaStream_t s, sem_mesh* m) {
  std::vector<int64_t> vert;
  int64_t E = 0;
  SEM_TRY(generator_vertices(d, vert, E));
  Topology topo;
  SEM_TRY(build_numbering(E, d.N, vert.data(), topo));
  std::vector<uint8_t> dface;
  generator_dirichlet(d, E, dface);
  GsPlan plan;
  SEM_TRY(build_gs_plan(topo, dface.data(), plan));
  m->dface = dface;
  vert.clear();
  vert.shrink_to_fit();

  const int N = d.N, n = N + 1;
  const int64_t n3 = (int64_t)n * n * n, P = E * n3;
  m->N = N;
  m->n = n;
  m->E = E;
  m->n_local = P;
  m->n_global = topo.n_global;
  m->n_seg = plan.n_nodes;
  m->n_seg_points = plan.n_points;
  for (int c = 0; c < kGsClasses; ++c) {
    m->gs_off[c] = plan.off[c];
    m->gs_cnt[c] = plan.cnt[c];
  }
  SEM_CUDA(cudaGetDevice(&m->device));

  std::vector<double> xi, w, D;
  gll(N, xi, w, D);
  std::vector<float> D32(n * n), D32lo(n * n);
  for (int q = 0; q < n * n; ++q) {
    D32[q] = (float)D[q];
    D32lo[q] = (float)(D[q] - (double)D32[q]);
  }
  // even-odd tables (D is centro-antisymmetric; n even only)
  const int hh = n / 2;
  std::vector<double> eo64((n % 2 == 0) ? 4 * hh * hh : 0);
  std::vector<float> eodf(eo64.size() * 2);
  for (int dir = 0; dir < 2 && n % 2 == 0; ++dir)
    for (int i = 0; i < hh; ++i)
      for (int l = 0; l < hh; ++l) {
        // dir 0: D[i][l], D[i][n-1-l]; dir 1 (D^T): D[l][i], D[n-1-l][i]
        const double x = dir == 0 ? D[i * n + l] : D[l * n + i];
        const double y = dir == 0 ? D[i * n + (n - 1 - l)] : D[(n - 1 - l) * n + i];
        const int q = (dir * hh + i) * hh + l;
        eo64[2 * q] = (x + y) / 2;
        eo64[2 * q + 1] = (x - y) / 2;
        for (int c = 0; c < 2; ++c) {
          const float hi = (float)eo64[2 * q + c];
          eodf[4 * q + 2 * c] = hi;
          eodf[4 * q + 2 * c + 1] = (float)(eo64[2 * q + c] - (double)hi);
        }
      }

  size_t& tb = m->dev_bytes;
  SEM_TRY(dev_alloc(&m->xyz, 3 * P, tb));
  SEM_TRY(dev_alloc(&m->G64, 6 * P, tb));
  SEM_TRY(dev_alloc(&m->B64, P, tb));
  SEM_TRY(dev_alloc(&m->G32, 6 * P, tb));
  SEM_TRY(dev_alloc(&m->G32lo, 6 * P, tb));
  SEM_TRY(dev_alloc(&m->B32, P, tb));
  SEM_TRY(dev_alloc(&m->B32lo, P, tb));
  SEM_TRY(dev_alloc(&m->dK, P, tb));
  SEM_TRY(dev_alloc(&m->dB, P, tb));
  SEM_TRY(dev_alloc(&m->wm, P, tb));
  SEM_TRY(dev_alloc(&m->gs_idx, plan.idx.size(), tb));
  SEM_TRY(dev_alloc(&m->gs_ptr, plan.gptr.size(), tb));
  SEM_TRY(dev_alloc(&m->gs_units, std::max<size_t>(plan.units.size(), 4), tb));
  m->gs_nunits = (int64_t)plan.units.size() / 4;
  SEM_TRY(dev_alloc(&m->D64, n * n, tb));
  SEM_TRY(dev_alloc(&m->dev_err, 1, tb));
  SEM_TRY(dev_alloc(&m->D32, n * n, tb));
  SEM_TRY(dev_alloc(&m->D32lo, n * n, tb));
  if (!eo64.empty()) {
    SEM_TRY(dev_alloc(&m->eo64, eo64.size(), tb));
    SEM_TRY(dev_alloc(&m->eodf, eodf.size(), tb));
  }

  size_t tmp_bytes = 0;
  double *xi_d = nullptr, *w_d = nullptr, *tlev_d = nullptr;
  int* bad_d = nullptr;
  struct Tmp {
    double** a;
    double** b;
    double** c;
    int** f;
    ~Tmp() {
      if (*a) cudaFree(*a);
      if (*b) cudaFree(*b);
      if (*c) cudaFree(*c);
      if (*f) cudaFree(*f);
    }
  } tmp{&xi_d, &w_d, &tlev_d, &bad_d};
  SEM_TRY(dev_alloc(&xi_d, n, tmp_bytes));
  SEM_TRY(dev_alloc(&w_d, n, tmp_bytes));
  SEM_TRY(dev_alloc(&bad_d, 1, tmp_bytes));

  SEM_CUDA(cudaMemcpyAsync(xi_d, xi.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaMemcpyAsync(w_d, w.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaMemcpyAsync(m->D64, D.data(), n * n * sizeof(double), cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaMemcpyAsync(m->D32, D32.data(), n * n * sizeof(float), cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaMemcpyAsync(m->D32lo, D32lo.data(), n * n * sizeof(float), cudaMemcpyHostToDevice, s));
  if (!eo64.empty()) {
    SEM_CUDA(cudaMemcpyAsync(m->eo64, eo64.data(), eo64.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    SEM_CUDA(cudaMemcpyAsync(m->eodf, eodf.data(), eodf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  SEM_CUDA(cudaMemsetAsync(bad_d, 0, sizeof(int), s));
  SEM_CUDA(cudaMemsetAsync(m->dev_err, 0, sizeof(int), s));
  SEM_CUDA(cudaMemcpyAsync(m->wm, plan.wm.data(), P, cudaMemcpyHostToDevice, s));
  if (!plan.idx.empty())
    SEM_CUDA(cudaMemcpyAsync(m->gs_idx, plan.idx.data(), plan.idx.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA(cudaMemcpyAsync(m->gs_ptr, plan.gptr.data(), plan.gptr.size() * 4, cudaMemcpyHostToDevice, s));
  if (!plan.units.empty())
    SEM_CUDA(cudaMemcpyAsync(m->gs_units, plan.units.data(), plan.units.size() * 4, cudaMemcpyHostToDevice, s));

  std::vector<double> tlev;
  if (d.kind == SEM_MESH_BOX) {
    launch_coords_box(m->xyz, xi_d, n, E, d.nx, d.ny, d.nz, d.lx, d.ly, d.lz, s);
  } else if (d.kind == SEM_MESH_PIPE) {
    tlev.resize(d.nr + 1);
    for (int k = 0; k <= d.nr; ++k) tlev[k] = 1.0 - std::tanh(d.beta * (1.0 - (double)k / d.nr)) / std::tanh(d.beta);
    SEM_TRY(dev_alloc(&tlev_d, d.nr + 1, tmp_bytes));
    SEM_CUDA(cudaMemcpyAsync(tlev_d, tlev.data(), tlev.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_coords_pipe(m->xyz, xi_d, tlev_d, n, E, d.nc, d.nr, d.nzp, d.R, d.L, d.a, s);
  } else {
    SEM_CUDA(cudaMemcpyAsync(m->xyz, d.xyz, 3 * P * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(launch_geometry(m->xyz, m->G64, m->B64, m->D64, w_d, n, E, bad_d, s));
  // assembled diagonals for the Jacobi preconditioner: dK = QQ^T diag(stiffness), dB = QQ^T B
  launch_local_diag(m->G64, m->dK, m->D64, n, E, s);
  SEM_CUDA(launch_gs<double>(m->dK, gs_dev(m), 0, nullptr, s));
  SEM_CUDA(cudaMemcpyAsync(m->dB, m->B64, P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SEM_CUDA(launch_gs<double>(m->dB, gs_dev(m), 0, nullptr, s));
  launch_split_f64(m->G64, m->G32, m->G32lo, 6 * P, s);
  launch_split_f64(m->B64, m->B32, m->B32lo, P, s);
  SEM_CUDA(cudaGetLastError());
  count_launches(7);
  int bad = 0;
  SEM_CUDA(cudaMemcpyAsync(&bad, bad_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    set_error("mesh has an element with det(J) <= 0");
    return SEM_ERR_BAD_MESH;
  }
  m->glo = std::move(topo.glo);
  return SEM_OK;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" {

const char* sem_last_error(void) { return g_last_error.c_str(); }

int sem_version(void) { return 1; }

int sem_mesh_fp64_kernel(const sem_mesh* m) { return m ? m->fp64_df : -1; }

int sem_mesh_ax_variant(const sem_mesh* m, sem_prec prec) {
  if (!m) return -1;
  if (prec == SEM_FP64) return m->fp64_df ? m->ax_var[2] : m->ax_var[0];
  if (prec == SEM_FP32) return m->ax_var[1];
  return -1;
}

sem_status sem_mesh_check(const sem_mesh* m, void* stream) {
  if (!m) {
    set_error("sem_mesh_check: null mesh");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  SEM_CUDA(cudaMemcpyAsync(&err, m->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA(cudaStreamSynchronize(s));
  if (err) {
    SEM_CUDA(cudaMemsetAsync(m->dev_err, 0, sizeof(int), s));
    SEM_CUDA(cudaStreamSynchronize(s));
    set_error("a bounded device-side wait of a local-operator kernel gave up; its output is invalid");
    return SEM_ERR_DEVICE_TIMEOUT;
  }
  return SEM_OK;
}

uint64_t sem_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* sem_status_str(sem_status s) {
  switch (s) {
    case SEM_OK: return "SEM_OK";
    case SEM_ERR_INVALID: return "SEM_ERR_INVALID";
    case SEM_ERR_OOM: return "SEM_ERR_OOM";
    case SEM_ERR_CUDA: return "SEM_ERR_CUDA";
    case SEM_ERR_NOT_CONVERGED: return "SEM_ERR_NOT_CONVERGED";
    case SEM_ERR_BREAKDOWN: return "SEM_ERR_BREAKDOWN";
    case SEM_ERR_BUSY: return "SEM_ERR_BUSY";
    case SEM_ERR_DEVICE_TIMEOUT: return "SEM_ERR_DEVICE_TIMEOUT";
    case SEM_ERR_BAD_MESH: return "SEM_ERR_BAD_MESH";
    case SEM_ERR_TIMEOUT: return "SEM_ERR_TIMEOUT";
    case SEM_ERR_NOT_FOUND: return "SEM_ERR_NOT_FOUND";
    case SEM_ERR_CANCELLED: return "SEM_ERR_CANCELLED";
  }
  return "SEM_ERR_UNKNOWN";
}

sem_status sem_mesh_create(const sem_mesh_desc* desc, void* stream, sem_mesh** out) {
  SEM_TRACE("sem_mesh_create");
  if (!desc || !out) {
    set_error("sem_mesh_create: null argument");
    return SEM_ERR_INVALID;
  }
  *out = nullptr;
  sem_mesh* m = new (std::nothrow) sem_mesh();
  if (!m) return SEM_ERR_OOM;
  sem_status st = build_mesh(*desc, (cudaStream_t)stream, m);
  if (st != SEM_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    free_mesh_arrays(m);
    delete m;
    return st;
  }
  st = autotune_mesh(m, (cudaStream_t)stream);
  if (st != SEM_OK) {
    free_mesh_arrays(m);
    delete m;
    return st;
  }
  *out = m;
  return SEM_OK;
}

sem_status sem_mesh_destroy(sem_mesh* m) {
  if (!m) return SEM_OK;
  // No device-wide synchronisation here: another thread may be capturing a
  // CUDA graph (the solvers and the batch engine do), and synchronising the
  // device while any stream captures is invalid.  The workspace's stream is
  // synchronised by release_workspace, and cudaFree waits for the work that
  // still uses the memory it frees.
  cudaSetDevice(m->device);
  release_workspace(m);
  free_mesh_arrays(m);
  delete m;
  return SEM_OK;
}

sem_status sem_mesh_set_coefficients(sem_mesh* m, const double* h1_dev, const double* h2_dev, void* stream) {
  SEM_TRACE("sem_mesh_set_coefficients");
  if (!m) {
    set_error("sem_mesh_set_coefficients: null mesh");
    return SEM_ERR_INVALID;
  }
  SEM_CUDA(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(m->ws_mutex);
  CoefArrays c;
  sem_status st = build_coef(m, h1_dev, h2_dev, c, s);
  if (st != SEM_OK) {
    cudaStreamSynchronize(s);
    c.release();
    return st;
  }
  // the old arrays are freed below: cudaFree waits for kernels still reading
  // them (no device-wide synchronisation, see sem_mesh_destroy)
  if (m->ws) SEM_CUDA(cudaStreamSynchronize(m->ws->s));
  m->dev_bytes -= coef_bytes(m);
  dev_free(m->cG64);
  dev_free(m->cG32);
  dev_free(m->cG32lo);
  dev_free(m->cdK);
  dev_free(m->cB64);
  dev_free(m->cB32);
  dev_free(m->cB32lo);
  dev_free(m->cdB);
  m->cG64 = c.G64;
  m->cG32 = c.G32;
  m->cG32lo = c.G32lo;
  m->cdK = c.dK;
  m->cB64 = c.B64;
  m->cB32 = c.B32;
  m->cB32lo = c.B32lo;
  m->cdB = c.dB;
  m->dev_bytes += coef_bytes(m);
  m->coef_gen++;
  if (m->ws) m->ws->minv_h1 = NAN;  // the cached Jacobi inverse belongs to the old operator
  return SEM_OK;
}

sem_status sem_mesh_info(const sem_mesh* m, sem_mesh_info_t* info) {
  if (!m || !info) {
    set_error("sem_mesh_info: null argument");
    return SEM_ERR_INVALID;
  }
  info->E = m->E;
  info->N = m->N;
  info->n_local = m->n_local;
  info->n_global = m->n_global;
  info->n_segments = m->n_seg;
  info->n_seg_points = m->n_seg_points;
  info->dev_bytes = m->dev_bytes;
  return SEM_OK;
}

sem_status sem_mesh_global_ids(const sem_mesh* m, int64_t* host_out) {
  if (!m || !host_out) {
    set_error("sem_mesh_global_ids: null argument");
    return SEM_ERR_INVALID;
  }
  std::memcpy(host_out, m->glo.data(), m->glo.size() * sizeof(int64_t));
  return SEM_OK;
}

sem_status sem_mesh_coords(const sem_mesh* m, double* xyz_dev, void* stream) {
  if (!m || !xyz_dev) {
    set_error("sem_mesh_coords: null argument");
    return SEM_ERR_INVALID;
  }
  SEM_CUDA(cudaMemcpyAsync(xyz_dev, m->xyz, 3 * m->n_local * sizeof(double), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return SEM_OK;
}

sem_status sem_mesh_geometry(const sem_mesh* m, double* G_dev, double* B_dev, void* stream) {
  if (!m) {
    set_error("sem_mesh_geometry: null mesh");
    return SEM_ERR_INVALID;
  }
  if (G_dev)
    SEM_CUDA(cudaMemcpyAsync(G_dev, m->G64, 6 * m->n_local * sizeof(double), cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  if (B_dev)
    SEM_CUDA(cudaMemcpyAsync(B_dev, m->B64, m->n_local * sizeof(double), cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  return SEM_OK;
}

sem_status sem_mesh_weights(const sem_mesh* m, double* mult_dev, double* mask_dev, void* stream) {
  if (!m) {
    set_error("sem_mesh_weights: null mesh");
    return SEM_ERR_INVALID;
  }
  launch_weights(m->wm, mult_dev, mask_dev, m->n_local, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  count_launches(1);
  return SEM_OK;
}

sem_status sem_ax(const sem_mesh* m, const void* u_dev, void* w_dev, double h1, double h2, sem_prec prec,
                  void* stream) {
  SEM_TRACE("sem_ax");
  if (!m || !u_dev || !w_dev) {
    set_error("sem_ax: null argument");
    return SEM_ERR_INVALID;
  }
  if (u_dev == w_dev) {
    set_error("sem_ax: u and w must not overlap");
    return SEM_ERR_INVALID;
  }
  return apply_local(m, u_dev, w_dev, h1, h2, prec, (cudaStream_t)stream);
}

sem_status sem_gs(const sem_mesh* m, void* v_dev, sem_prec prec, int apply_mask, void* stream) {
  SEM_TRACE("sem_gs");
  if (!m || !v_dev) {
    set_error("sem_gs: null argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SEM_FP64) {
    SEM_CUDA(launch_gs<double>((double*)v_dev, gs_dev(m), apply_mask, nullptr, s));
  } else if (prec == SEM_FP32) {
    SEM_CUDA(launch_gs<float>((float*)v_dev, gs_dev(m), apply_mask, nullptr, s));
  } else {
    set_error("sem_gs: prec must be SEM_FP64 or SEM_FP32");
    return SEM_ERR_INVALID;
  }
  count_launches(1);
  return SEM_OK;
}

sem_status sem_rhs(const sem_mesh* m, const double* f_dev, double* b_dev, void* stream) {
  SEM_TRACE("sem_rhs");
  if (!m || !f_dev || !b_dev) {
    set_error("sem_rhs: null argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  launch_mul(b_dev, m->B64, f_dev, m->n_local, s);
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(launch_gs<double>(b_dev, gs_dev(m), 1, nullptr, s));
  count_launches(2);
  return SEM_OK;
}

sem_status sem_apply(const sem_mesh* m, const double* x_dev, double* y_dev, double h1, double h2, void* stream) {
  SEM_TRACE("sem_apply");
  if (!m || !x_dev || !y_dev || x_dev == y_dev) {
    set_error("sem_apply: null or overlapping argument");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  sem_status st = apply_local(m, x_dev, y_dev, h1, h2, SEM_FP64, s);
  if (st != SEM_OK) return st;
  SEM_CUDA(launch_gs<double>(y_dev, gs_dev(m), 1, nullptr, s));
  count_launches(1);
  return SEM_OK;
}

sem_status sem_jacobi(const sem_mesh* m, double h1, double h2, double* minv_dev, void* stream) {
  SEM_TRACE("sem_jacobi");
  if (!m || !minv_dev) {
    set_error("sem_jacobi: null argument");
    return SEM_ERR_INVALID;
  }
  launch_minv(minv_dev, nullptr, m->opdK(), m->opdB(), m->wm, h1, h2, m->n_local, (cudaStream_t)stream);
  SEM_CUDA(cudaGetLastError());
  count_launches(1);
  return SEM_OK;
}

sem_status sem_topology_numbering(int64_t E, int N, const int64_t* vert, int64_t* glo_host, int64_t* n_global) {
  SEM_TRACE("sem_topology_numbering");
  if (!vert || !glo_host) {
    set_error("sem_topology_numbering: null argument");
    return SEM_ERR_INVALID;
  }
  Topology t;
  sem_status st = build_numbering(E, N, vert, t);
  if (st != SEM_OK) return st;
  std::memcpy(glo_host, t.glo.data(), t.glo.size() * sizeof(int64_t));
  if (n_global) *n_global = t.n_global;
  return SEM_OK;
}

sem_status sem_mesh_vertices(const sem_mesh_desc* desc, int64_t* vert_host, int64_t* E_out) {
  if (!desc) {
    set_error("sem_mesh_vertices: null descriptor");
    return SEM_ERR_INVALID;
  }
  std::vector<int64_t> vert;
  int64_t E = 0;
  sem_status st = generator_vertices(*desc, vert, E);
  if (st != SEM_OK) return st;
  if (E_out) *E_out = E;
  if (vert_host) std::memcpy(vert_host, vert.data(), vert.size() * sizeof(int64_t));
  return SEM_OK;
}

}  // extern "C"
