// Projection onto previous solutions for successive solves with one operator
// (Sec. 2: the velocity and pressure solves start from the projection of the
// new solution onto the space of earlier ones; the paper cites Fischer 1998).
//
// The space is an A-orthonormal basis X = [x_1 .. x_l] of earlier solutions
// (global inner product <a, b> = sum_q a_q b_q / mult_q on local vectors) and
// AX = [A x_1 .. A x_l], kept on the device.  A solve
//   1. forms xbar = sum_i <x_i, b> x_i, the A-norm best approximation to
//      A^{-1} b from the space (coefficients stay on the device);
//   2. runs the library's PCG from xbar (sem_pcg_solve, any precision);
//   3. A-orthogonalises v = x - xbar against X by two classical Gram-Schmidt
//      passes (coefficients <A x_i, v>), computes A v with the native FP64
//      operator, and appends v / ||v||_A and A v / ||v||_A; a full basis
//      restarts from x alone.
// All reductions are deterministic: per-block partials summed in a fixed
// order by a second kernel.
#include <cmath>
#include <cstring>
#include <new>

#include "kernels.h"
#include "sem_internal.h"
#include "solver.h"

struct sem_proj {
  sem_mesh* m = nullptr;
  int L = 0, l = 0;
  double h1 = 1.0, h2 = 0.0;
  uint64_t coef_gen = 0;   // the mesh's coefficient generation the basis belongs to
  int64_t n = 0;
  double* X = nullptr;     // [L][n]
  double* AX = nullptr;    // [L][n]
  double* xbar = nullptr;  // [n]
  double* v = nullptr;     // [n]
  double* Av = nullptr;    // [n]
  double* part = nullptr;  // [kBlocks][kMaxV] block partials
  double* coef = nullptr;  // [kMaxV + 1]: Gram-Schmidt / projection coefficients, then <v, A v>
  double* nrm_h = nullptr; // pinned copy of <v, A v>
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace sem {
namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 4;
constexpr int kMaxV = SEM_PROJ_MAX_VECTORS;

__device__ __forceinline__ void fill_inv(double* sinv) {
  for (int m = threadIdx.x; m < 128; m += blockDim.x) sinv[m] = m ? 1.0 / (double)m : 0.0;
}

// part[b][i] = block b's share of <V_i, y> for i < nv
__global__ void __launch_bounds__(kThreads) k_mdot(const double* __restrict__ V, int nv, const double* __restrict__ y,
                                                   const uint8_t* __restrict__ wm, int64_t n, double* __restrict__ part) {
  __shared__ double sred[32];
  __shared__ double sinv[128];
  fill_inv(sinv);
  __syncthreads();
  double acc[kMaxV];
#pragma unroll
  for (int i = 0; i < kMaxV; ++i) acc[i] = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads) {
    const double yq = y[q] * sinv[wm[q] & 0x7f];
#pragma unroll
    for (int i = 0; i < kMaxV; ++i)
      if (i < nv) acc[i] = fma(V[i * n + q], yq, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < kMaxV; ++i) {
    if (i >= nv) break;
    const double s = block_sum(acc[i], sred);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxV + i] = s;
  }
}

// out[i] = sum over blocks of part[.][i], in block order (one CTA per i)
__global__ void __launch_bounds__(kThreads) k_mfinal(const double* __restrict__ part, int nblocks, double* out) {
  __shared__ double sred[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) s += part[b * kMaxV + i];
  s = block_sum(s, sred);
  if (threadIdx.x == 0) out[i] = s;
}

// y = base - sum_{i < nv} c_i V_i   (base may alias y), or y = sum c_i V_i when base is null
__global__ void __launch_bounds__(kThreads) k_combo(double* y, const double* base, const double* __restrict__ V, int nv,
                                                    const double* __restrict__ c, int64_t n) {
  __shared__ double sc[kMaxV];
  if (threadIdx.x < kMaxV) sc[threadIdx.x] = threadIdx.x < nv ? c[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kMaxV; ++i)
      if (i < nv) s = fma(sc[i], V[i * n + q], s);
    y[q] = base ? base[q] - s : s;
  }
}

// y = a x + b z (z may be null)
__global__ void __launch_bounds__(kThreads) k_axpby(double* y, double a, const double* __restrict__ x, double b,
                                                    const double* __restrict__ z, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kThreads)
    y[q] = z ? a * x[q] + b * z[q] : a * x[q];
}

// coef[0..nv) = <V_i, y>
cudaError_t mdot(sem_proj* p, const double* V, int nv, const double* y, double* out, cudaStream_t s) {
  k_mdot<<<kBlocks, kThreads, 0, s>>>(V, nv, y, p->m->wm, p->n, p->part);
  k_mfinal<<<nv, kThreads, 0, s>>>(p->part, kBlocks, out);
  count_launches(2);
  return cudaGetLastError();
}

void free_proj(sem_proj* p) {
  for (double* d : {p->X, p->AX, p->xbar, p->v, p->Av, p->part, p->coef})
    if (d) cudaFree(d);
  if (p->nrm_h) cudaFreeHost(p->nrm_h);
  if (p->e0) cudaEventDestroy(p->e0);
  if (p->e1) cudaEventDestroy(p->e1);
  delete p;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" {

sem_status sem_proj_create(const sem_mesh* mesh, int max_vectors, double h1, double h2, sem_proj** out) {
  if (!mesh || !out) {
    set_error("sem_proj_create: null argument");
    return SEM_ERR_INVALID;
  }
  *out = nullptr;
  if (max_vectors < 1 || max_vectors > SEM_PROJ_MAX_VECTORS) {
    set_error("sem_proj_create: max_vectors must be in 1..SEM_PROJ_MAX_VECTORS");
    return SEM_ERR_INVALID;
  }
  if (!(h1 >= 0.0) || !(h2 >= 0.0) || (h1 == 0.0 && h2 == 0.0)) {
    set_error("sem_proj_create: need h1 >= 0, h2 >= 0, not both zero");
    return SEM_ERR_INVALID;
  }
  SEM_CUDA(cudaSetDevice(mesh->device));
  sem_proj* p = new (std::nothrow) sem_proj();
  if (!p) return SEM_ERR_OOM;
  p->m = const_cast<sem_mesh*>(mesh);
  p->L = max_vectors;
  p->h1 = h1;
  p->h2 = h2;
  p->coef_gen = mesh->coef_gen;
  p->n = mesh->n_local;
  const size_t vb = (size_t)p->n * sizeof(double);
  cudaError_t e = cudaMalloc((void**)&p->X, vb * max_vectors);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->AX, vb * max_vectors);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->xbar, vb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->v, vb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->Av, vb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->part, sizeof(double) * kBlocks * kMaxV);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->coef, sizeof(double) * (kMaxV + 1));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->nrm_h, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&p->e0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->e1);
  if (e != cudaSuccess) {
    free_proj(p);
    cudaGetLastError();
    set_error(std::string("sem_proj_create: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA;
  }
  *out = p;
  return SEM_OK;
}

sem_status sem_proj_destroy(sem_proj* p) {
  if (!p) return SEM_OK;
  cudaSetDevice(p->m->device);
  free_proj(p);  // cudaFree waits for work still using the space (no device-wide sync: see sem_mesh_destroy)
  return SEM_OK;
}

sem_status sem_proj_size(const sem_proj* p, int* nvec) {
  if (!p || !nvec) {
    set_error("sem_proj_size: null argument");
    return SEM_ERR_INVALID;
  }
  *nvec = p->l;
  return SEM_OK;
}

sem_status sem_proj_reset(sem_proj* p) {
  if (!p) {
    set_error("sem_proj_reset: null argument");
    return SEM_ERR_INVALID;
  }
  p->l = 0;
  return SEM_OK;
}

sem_status sem_proj_solve(sem_proj* p, const double* b_dev, double* x_dev, const sem_solve_opts* opts,
                          sem_solve_result* result, void* stream) {
  SEM_TRACE("sem_proj_solve");
  if (!p || !b_dev || !x_dev || !opts) {
    set_error("sem_proj_solve: null argument");
    return SEM_ERR_INVALID;
  }
  if (opts->h1 != p->h1 || opts->h2 != p->h2) {
    set_error("sem_proj_solve: opts->h1, h2 differ from the projection space's operator");
    return SEM_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  sem_mesh* m = p->m;
  if (p->coef_gen != m->coef_gen) {  // new per-point coefficients: the basis is no longer A-orthonormal
    p->l = 0;
    p->coef_gen = m->coef_gen;
  }
  const int64_t n = p->n;
  const size_t vb = (size_t)n * sizeof(double);
  SEM_CUDA(cudaEventRecord(p->e0, s));

  // 1. xbar = sum_i <x_i, b> x_i
  if (p->l > 0) {
    SEM_CUDA(mdot(p, p->X, p->l, b_dev, p->coef, s));
    k_combo<<<kBlocks, kThreads, 0, s>>>(p->xbar, nullptr, p->X, p->l, p->coef, n);
    count_launches(1);
  } else {
    SEM_CUDA(cudaMemsetAsync(p->xbar, 0, vb, s));
  }
  SEM_CUDA(cudaMemcpyAsync(x_dev, p->xbar, vb, cudaMemcpyDeviceToDevice, s));

  // 2. PCG from xbar
  sem_solve_result r;
  std::memset(&r, 0, sizeof(r));
  sem_status st = sem_pcg_solve(m, b_dev, x_dev, opts, &r, stream);
  if (st == SEM_OK) {
    // 3. the new direction, A-orthogonal to the basis
    if (p->l >= p->L) {  // full: restart from x alone
      p->l = 0;
      SEM_CUDA(cudaMemcpyAsync(p->v, x_dev, vb, cudaMemcpyDeviceToDevice, s));
    } else {
      k_axpby<<<kBlocks, kThreads, 0, s>>>(p->v, 1.0, x_dev, -1.0, p->xbar, n);
      count_launches(1);
    }
    for (int pass = 0; pass < 2 && p->l > 0; ++pass) {
      SEM_CUDA(mdot(p, p->AX, p->l, p->v, p->coef, s));
      k_combo<<<kBlocks, kThreads, 0, s>>>(p->v, p->v, p->X, p->l, p->coef, n);
      count_launches(1);
    }
    SEM_CUDA(ax64_exact(m, p->v, p->Av, p->h1, p->h2, s));
    SEM_CUDA(launch_gs<double>(p->Av, gs_dev(m), 1, nullptr, s));
    count_launches(2);
    SEM_CUDA(mdot(p, p->v, 1, p->Av, p->coef + kMaxV, s));
    SEM_CUDA(cudaMemcpyAsync(p->nrm_h, p->coef + kMaxV, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    const double nrm2 = *p->nrm_h;
    if (nrm2 > 0.0 && std::isfinite(nrm2)) {  // nothing to add when b was already in the space
      const double sc = 1.0 / std::sqrt(nrm2);
      k_axpby<<<kBlocks, kThreads, 0, s>>>(p->X + (size_t)p->l * n, sc, p->v, 0.0, nullptr, n);
      k_axpby<<<kBlocks, kThreads, 0, s>>>(p->AX + (size_t)p->l * n, sc, p->Av, 0.0, nullptr, n);
      count_launches(2);
      p->l += 1;
    }
  }
  SEM_CUDA(cudaGetLastError());
  SEM_CUDA(cudaEventRecord(p->e1, s));
  SEM_CUDA(cudaEventSynchronize(p->e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->e0, p->e1);
  r.ms = ms;
  if (result) *result = r;
  return st;
}

}  // extern "C"
