// sem_pcg_solve_noalloc: the FP64 Jacobi-PCG solve of sem_pcg_solve for callers
// that cannot allocate device memory.  It follows sem_pcg_solve's FP64 rule:
// CG on the tuned operator, then the true residual with the native FP64
// operator and restarts from x while that residual misses the tolerance;
// result->rel_res is that true residual.
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns every byte of the device (a fixed pool handed out up front),
// real-time loops where an allocation's latency or implicit device-wide
// synchronisation is not acceptable, and plug-ins whose host process forbids
// allocations outside its own allocator.  sem_pcg_solve keeps its scratch
// (work vectors, reduction partials, the device-side CG state) in a
// workspace it allocates on first use; this entry point keeps that scratch in
// one file-scope device array of fixed size instead, and allocates nothing.
//
// Limits and sharing (also stated in include/sem.h):
//   * n_local <= SEM_NOALLOC_MAX_POINTS local points;
//   * the array is shared by every call in the process, on this device: calls
//     that overlap on the GPU race with each other and give wrong results;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress; make that first call before any stream capture.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "sem_internal.h"
#include "solver.h"

namespace sem {
namespace {

constexpr int64_t kMaxPoints = SEM_NOALLOC_MAX_POINTS;
constexpr int kVectors = 5;  // r, z, p, w, M^{-1}
constexpr int64_t kMaxAxPartials = kMaxPoints / 8;  // >= ceil(E / elems-per-block) for every N >= 1
constexpr int64_t kStateDoubles = (sizeof(PcgState) + sizeof(double) - 1) / sizeof(double);
constexpr int64_t kScratchDoubles = kVectors * kMaxPoints + kMaxAxPartials + 3 * 1024 + kStateDoubles;

// All scratch of the no-allocation solve (about 10.5 MB).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of the array for the current device (looked up once per device).
sem_status scratch_address(double** out) {
  int dev = 0;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sem_pcg_solve_noalloc: device ordinal out of range");
    return SEM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return SEM_OK;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" sem_status sem_pcg_solve_noalloc(const sem_mesh* m, const double* b_dev, double* x_dev,
                                            const sem_solve_opts* opts, sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_pcg_solve_noalloc");
  if (!m || !b_dev || !x_dev || !opts) {
    set_error("sem_pcg_solve_noalloc: null argument");
    return SEM_ERR_INVALID;
  }
  if (m->n_local > kMaxPoints) {
    set_error("sem_pcg_solve_noalloc: mesh has " + std::to_string(m->n_local) +
              " local points, more than SEM_NOALLOC_MAX_POINTS = " + std::to_string(kMaxPoints));
    return SEM_ERR_INVALID;
  }
  if (((uintptr_t)b_dev | (uintptr_t)x_dev) & 15u) {
    set_error("sem_pcg_solve_noalloc: b_dev and x_dev must be 16-byte aligned");
    return SEM_ERR_INVALID;
  }
  if (opts->prec != SEM_FP64) {
    set_error("sem_pcg_solve_noalloc: only prec = SEM_FP64 is supported");
    return SEM_ERR_INVALID;
  }
  const double h1 = opts->h1, h2 = opts->h2;
  if (!(h1 >= 0.0) || !(h2 >= 0.0) || (h1 == 0.0 && h2 == 0.0)) {
    set_error("sem_pcg_solve_noalloc: need h1 >= 0, h2 >= 0, not both zero");
    return SEM_ERR_INVALID;
  }
  const double tol = opts->tol > 0.0 ? opts->tol : 1e-10;
  const int maxit = opts->maxit > 0 ? opts->maxit : 20000;
  cudaStream_t s = (cudaStream_t)stream;

  // the mesh's device (each device has its own copy of the array), and the
  // kernel choice, which the autotuner writes under the mesh's lock
  SEM_CUDA(cudaSetDevice(m->device));
  sem_mesh* mm = const_cast<sem_mesh*>(m);
  int var_native = 0, var_df = 0, use_df = 0;
  {
    std::lock_guard<std::mutex> lk(mm->ws_mutex);
    var_native = m->ax_var[0];
    var_df = m->ax_var_dff;  // the fused form runs here
    use_df = m->fp64_df;
  }

  double* base = nullptr;
  sem_status st = scratch_address(&base);
  if (st != SEM_OK) return st;
  const int64_t n = m->n_local;
  double* r = base;
  double* z = r + kMaxPoints;
  double* p = z + kMaxPoints;
  double* w = p + kMaxPoints;
  double* minv = w + kMaxPoints;
  double* part_ax = minv + kMaxPoints;
  double* part_vec = part_ax + kMaxAxPartials;
  PcgState* dst = reinterpret_cast<PcgState*>(part_vec + 3 * 1024);

  launch_mask(x_dev, m->wm, n, s);
  launch_minv(minv, nullptr, m->opdK(), m->opdB(), m->wm, h1, h2, n, s);
  count_launches(2);
  VecParams<double> v{x_dev, r, z, p, w, minv, b_dev, m->wm, n, dst, part_vec};

  // the fused CG operator: the tuned kernel (double-float or native FP64)
  auto fused_ax = [&]() -> cudaError_t {
    if (use_df) {
      AxDFParams a{nullptr, w, m->opG32(), m->opG32lo(), m->opB32(), m->opB32lo(), m->D32, m->D32lo, h1, h2,
                   h2 != 0.0, m->E, z, p, dst, part_ax, m->eo64, m->eodf};
      return launch_ax_df(m->N, var_df, true, a, s, nullptr);
    }
    AxParams<double> a{nullptr, w, m->opG64(), m->opB64(), m->D64, h1, h2, h2 != 0.0, m->E, z, p, dst, part_ax,
                       m->dev_err};
    return launch_ax_f64(m->N, var_native, true, a, s, nullptr);
  };

  // The same rule as sem_pcg_solve's FP64 solve: CG runs on its recurrences;
  // once they meet the tolerance, the true residual b - A x is formed with
  // the native FP64 operator (exact FP64 arithmetic), and CG restarts from x
  // if that residual misses (at most kMaxRestarts times within maxit).
  constexpr int kMaxRestarts = 3;
  constexpr int kChunk = 8;
  int iters = 0, passes = 0;
  double rel = 0.0;
  sem_status status = SEM_OK;
  for (int pass = 0;; ++pass) {
    // The array keeps the previous call's contents: the state (reduction
    // counters included) is written in full before any kernel reads it.
    PcgState h;
    std::memset(&h, 0, sizeof(h));
    h.tol2 = tol * tol;
    h.maxit = maxit - iters;
    SEM_CUDA(cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    SEM_CUDA(ax64_exact(m, x_dev, w, h1, h2, s));
    SEM_CUDA(launch_gs<double>(w, gs_dev(m), 1, nullptr, s));
    SEM_CUDA(launch_residual(r, b_dev, w, m->wm, n, dst, part_vec, 1, s));
    SEM_CUDA(launch_pcg_init<double>(v, s));
    count_launches(4);
    PcgState cur;
    SEM_CUDA(cudaMemcpyAsync(&cur, dst, sizeof(cur), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    if (cur.bb == 0.0) {  // b = 0: x = 0
      SEM_CUDA(cudaMemsetAsync(x_dev, 0, n * sizeof(double), s));
      SEM_CUDA(cudaStreamSynchronize(s));
      rel = 0.0;
      status = SEM_OK;
      break;
    }
    rel = std::sqrt(cur.aux / cur.bb);  // true residual of the current x
    passes = pass;
    if (rel <= tol) {
      status = SEM_OK;
      break;
    }
    if (pass > kMaxRestarts || iters >= maxit) {
      status = SEM_ERR_NOT_CONVERGED;
      break;
    }
    const int max_chunks = (maxit - iters) / kChunk + 2;
    for (int c = 0; c < max_chunks && !cur.done; ++c) {
      for (int k = 0; k < kChunk; ++k) {
        SEM_CUDA(fused_ax());
        SEM_CUDA(launch_gs<double>(w, gs_dev(m), 1, dst, s));
        SEM_CUDA(launch_pcg_update<double>(v, s));
      }
      count_launches(3 * kChunk);
      SEM_CUDA(cudaMemcpyAsync(&cur, dst, sizeof(cur), cudaMemcpyDeviceToHost, s));
      SEM_CUDA(cudaStreamSynchronize(s));
    }
    if (!cur.done) {
      set_error("sem_pcg_solve_noalloc: CG did not report completion within maxit iterations");
      return SEM_ERR_DEVICE_TIMEOUT;
    }
    iters += cur.iter;
    if (cur.status != SEM_OK) {  // breakdown, or maxit without meeting the tolerance
      rel = std::sqrt(cur.rr / cur.bb);
      status = (sem_status)cur.status;
      break;
    }
  }
  if (result) {
    result->iters = iters;
    result->outer_iters = passes;
    result->rel_res = rel;
    result->ms = 0.0;
    result->status = status;
  }
  return status;
}
