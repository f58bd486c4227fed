// Vector kernels of Jacobi-preconditioned CG with the inner products reduced
// on the device (Sec. 3: reductions as hand-written kernels instead of
// compiler-generated ones; scalars stay in device memory between kernels).
//
// Weighted inner product over local points: <a, b> = sum_l a_l b_l / mult_l,
// which equals the plain dot product over global nodes.  Every grid
// reduction is deterministic: fixed per-thread ranges, fixed block trees and
// a fixed-order sum of the block partials by the last block to arrive.
#include "kernels.h"

namespace sem {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 152 * 4;

int vec_grid() { return kVecBlocks; }

// FP64 accumulator.
struct Acc64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};

// FP32 products accumulated in double-float (Neumaier's compensated sum on
// the FP32 pipe), handed to the FP64 block reduction at the end.
struct AccF32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    c = __fadd_rn(c, err);
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

template <typename T>
struct AccOf;
template <>
struct AccOf<double> {
  using type = Acc64;
};
template <>
struct AccOf<float> {
  using type = AccF32;
};

template <typename T>
__device__ __forceinline__ void fill_inv_mult(T* sinv) {
  for (int m = threadIdx.x; m < 128; m += blockDim.x) sinv[m] = m ? T(1) / T(m) : T(0);
}

// x += alpha p; r -= alpha w; z = M^{-1} r; then <r, z>, <r, r>; the last block
// checks ||r|| <= tol ||b||, else forms beta = <r,z>_new / <r,z>_old.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_pcg_update(const VecParams<T> P) {
  using Acc = typename AccOf<T>::type;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  __shared__ int sdone;
  if (threadIdx.x == 0) sdone = P.st->done;
  fill_inv_mult(sinv);
  __syncthreads();
  if (sdone) return;
  const T alpha = (T)P.st->alpha;
  Acc rz, rr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.n; q += (int64_t)gridDim.x * blockDim.x) {
    const T pq = P.p[q], wq = P.w[q];
    const T rq = P.r[q] - alpha * wq;
    P.x[q] = P.x[q] + alpha * pq;
    P.r[q] = rq;
    const T zq = P.minv[q] * rq;
    P.z[q] = zq;
    const T im = sinv[P.wm[q] & 0x7f];
    rz.add(rq * zq * im);
    rr.add(rq * rq * im);
  }
  const double srz = block_sum(rz.get(), sred);
  const double srr = block_sum(rr.get(), sred);
  if (threadIdx.x == 0) {
    P.partial[2 * blockIdx.x] = srz;
    P.partial[2 * blockIdx.x + 1] = srr;
  }
  if (last_block(&P.st->cnt[1])) {
    const double rz_t = sum_partials(P.partial, gridDim.x, 2, 0, sred);
    const double rr_t = sum_partials(P.partial, gridDim.x, 2, 1, sred);
    if (threadIdx.x == 0) {
      PcgState* st = P.st;
      st->iter += 1;
      st->rr = rr_t;
      if (rr_t != rr_t || rz_t != rz_t) {
        st->done = 1;
        st->status = 5;  // SEM_ERR_BREAKDOWN (NaN)
      } else if (rr_t <= st->tol2 * st->bb) {
        st->done = 1;
        st->status = 0;
      } else if (st->iter >= st->maxit) {
        st->done = 1;
        st->status = 4;  // SEM_ERR_NOT_CONVERGED
      } else {
        st->beta = rz_t / st->rho;
        st->rho = rz_t;
      }
      st->cnt[1] = 0;
    }
  }
}

// Start of a CG run on residual r (already b - A x0) and right-hand side b:
// z = M^{-1} r, p = 0, rho = <r,z>, rr = <r,r>, bb = <b,b>, beta = 0.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_pcg_init(const VecParams<T> P) {
  using Acc = typename AccOf<T>::type;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  fill_inv_mult(sinv);
  __syncthreads();
  Acc rz, rr, bb;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.n; q += (int64_t)gridDim.x * blockDim.x) {
    const T rq = P.r[q], bq = P.b[q];
    const T zq = P.minv[q] * rq;
    P.z[q] = zq;
    P.p[q] = T(0);
    const T im = sinv[P.wm[q] & 0x7f];
    rz.add(rq * zq * im);
    rr.add(rq * rq * im);
    bb.add(bq * bq * im);
  }
  const double a = block_sum(rz.get(), sred);
  const double b = block_sum(rr.get(), sred);
  const double c = block_sum(bb.get(), sred);
  if (threadIdx.x == 0) {
    P.partial[3 * blockIdx.x] = a;
    P.partial[3 * blockIdx.x + 1] = b;
    P.partial[3 * blockIdx.x + 2] = c;
  }
  if (last_block(&P.st->cnt[2])) {
    const double rz_t = sum_partials(P.partial, gridDim.x, 3, 0, sred);
    const double rr_t = sum_partials(P.partial, gridDim.x, 3, 1, sred);
    const double bb_t = sum_partials(P.partial, gridDim.x, 3, 2, sred);
    if (threadIdx.x == 0) {
      PcgState* st = P.st;
      st->rho = rz_t;
      st->rr = rr_t;
      st->bb = bb_t;
      st->beta = 0.0;
      st->alpha = 0.0;
      st->iter = 0;
      st->status = 0;
      st->done = (bb_t == 0.0) || (rr_t <= st->tol2 * bb_t);
      st->cnt[2] = 0;
    }
  }
}

template <typename T>
cudaError_t launch_pcg_update(const VecParams<T>& p, cudaStream_t s) {
  k_pcg_update<T><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pcg_init(const VecParams<T>& p, cudaStream_t s) {
  k_pcg_init<T><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_pcg_update<double>(const VecParams<double>&, cudaStream_t);
template cudaError_t launch_pcg_update<float>(const VecParams<float>&, cudaStream_t);
template cudaError_t launch_pcg_init<double>(const VecParams<double>&, cudaStream_t);
template cudaError_t launch_pcg_init<float>(const VecParams<float>&, cudaStream_t);

// ---- small helpers ------------------------------------------------------------

#define GRID_STRIDE(q, n) \
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (n); q += (int64_t)gridDim.x * blockDim.x)

__global__ void k_mul(double* out, const double* a, const double* b, int64_t n) {
  GRID_STRIDE(q, n) out[q] = a[q] * b[q];
}
void launch_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t s) {
  k_mul<<<kVecBlocks, kVecThreads, 0, s>>>(out, a, b, n);
}

__global__ void k_mask(double* x, const uint8_t* wm, int64_t n) {
  GRID_STRIDE(q, n) if (wm[q] & 0x80) x[q] = 0.0;
}
void launch_mask(double* x, const uint8_t* wm, int64_t n, cudaStream_t s) {
  k_mask<<<kVecBlocks, kVecThreads, 0, s>>>(x, wm, n);
}

__global__ void k_minv(double* minv, float* minv32, const double* dK, const double* dB, const uint8_t* wm, double h1,
                       double h2, int64_t n) {
  GRID_STRIDE(q, n) {
    const double v = (wm[q] & 0x80) ? 0.0 : 1.0 / (h1 * dK[q] + h2 * dB[q]);
    minv[q] = v;
    if (minv32) minv32[q] = __double2float_rn(v);
  }
}
void launch_minv(double* minv, float* minv32, const double* dK, const double* dB, const uint8_t* wm, double h1,
                 double h2, int64_t n, cudaStream_t s) {
  k_minv<<<kVecBlocks, kVecThreads, 0, s>>>(minv, minv32, dK, dB, wm, h1, h2, n);
}

__global__ void __launch_bounds__(kVecThreads) k_residual(double* r, const double* b, const double* w,
                                                          const uint8_t* wm, int64_t n, PcgState* st,
                                                          double* partial, int set_bb) {
  __shared__ double sred[32];
  __shared__ double sinv[128];
  fill_inv_mult(sinv);
  __syncthreads();
  double rr = 0.0, bb = 0.0;
  GRID_STRIDE(q, n) {
    const double bq = b[q];
    const double rq = bq - w[q];
    r[q] = rq;
    const double im = sinv[wm[q] & 0x7f];
    rr += rq * rq * im;
    if (set_bb) bb += bq * bq * im;
  }
  const double a = block_sum(rr, sred);
  const double c = block_sum(bb, sred);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  if (last_block(&st->cnt[3])) {
    const double rr_t = sum_partials(partial, gridDim.x, 2, 0, sred);
    const double bb_t = sum_partials(partial, gridDim.x, 2, 1, sred);
    if (threadIdx.x == 0) {
      st->aux = rr_t;
      if (set_bb) st->bb = bb_t;
      st->cnt[3] = 0;
    }
  }
}
cudaError_t launch_residual(double* r, const double* b, const double* w, const uint8_t* wm, int64_t n, PcgState* st,
                            double* partial, int set_bb, cudaStream_t s) {
  k_residual<<<kVecBlocks, kVecThreads, 0, s>>>(r, b, w, wm, n, st, partial, set_bb);
  return cudaGetLastError();
}

__global__ void k_scale_to_f32(float* r32, const double* r, double sc, int64_t n) {
  GRID_STRIDE(q, n) r32[q] = __double2float_rn(r[q] * sc);
}
void launch_scale_to_f32(float* r32, const double* r, double sc, int64_t n, cudaStream_t s) {
  k_scale_to_f32<<<kVecBlocks, kVecThreads, 0, s>>>(r32, r, sc, n);
}

__global__ void k_accumulate(double* x, const float* d32, double sc, int64_t n) {
  GRID_STRIDE(q, n) x[q] += sc * (double)d32[q];
}
void launch_accumulate(double* x, const float* d32, double sc, int64_t n, cudaStream_t s) {
  k_accumulate<<<kVecBlocks, kVecThreads, 0, s>>>(x, d32, sc, n);
}

__global__ void k_zero_f32(float* a, int64_t n) {
  GRID_STRIDE(q, n) a[q] = 0.f;
}
void launch_zero_f32(float* a, int64_t n, cudaStream_t s) { k_zero_f32<<<kVecBlocks, kVecThreads, 0, s>>>(a, n); }

}  // namespace sem
