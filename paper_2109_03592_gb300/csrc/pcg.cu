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

// 16-byte vectors of T and the matching multiplicity bytes.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  using M = uchar4;
  static constexpr int W = 4;
  __device__ static float get(const V& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
  __device__ static void set(V& v, int k, float a) {
    if (k == 0) v.x = a; else if (k == 1) v.y = a; else if (k == 2) v.z = a; else v.w = a;
  }
  __device__ static unsigned char getm(const M& m, int k) { return k == 0 ? m.x : k == 1 ? m.y : k == 2 ? m.z : m.w; }
};
template <>
struct Vec16<double> {
  using V = double2;
  using M = uchar2;
  static constexpr int W = 2;
  __device__ static double get(const V& v, int k) { return k == 0 ? v.x : v.y; }
  __device__ static void set(V& v, int k, double a) {
    if (k == 0) v.x = a; else v.y = a;
  }
  __device__ static unsigned char getm(const M& m, int k) { return k == 0 ? m.x : m.y; }
};

// x += alpha p; r -= alpha w; z = M^{-1} r; then <r, z>, <r, r>; the last block
// checks ||r|| <= tol ||b||, else forms beta = <r,z>_new / <r,z>_old.
// Each thread moves 16-byte vectors (4 floats / 2 doubles per array), so a
// resident block keeps 5 x 16 B loads per thread in flight.
// EXT (a preconditioner applied by other kernels, e.g. overlapping Schwarz):
// only x, r and <r, r> with the stop tests here; z = M^{-1} r and beta come
// from the preconditioner's kernels and k_pcg_rho afterwards.
// XM: how x is advanced.  0: x += alpha p.  1: not at all (the first of a
// pair of iterations: alpha is kept in the state as alpha_prev and xpend
// set).  2: x += alpha_prev p2 + alpha p (the second of the pair, p2 the
// first's direction).  Pairing the x updates saves one read and one write of
// x per two iterations; k_pcg_xflush completes a pair cut short by a pause.
template <typename T, bool EXT, int XM>
__global__ void __launch_bounds__(kVecThreads) k_pcg_update(const VecParams<T> P) {
  using Acc = typename AccOf<T>::type;
  using VT = Vec16<T>;
  using V = typename VT::V;
  using M = typename VT::M;
  constexpr int W = VT::W;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  __shared__ int sdone;
  if (threadIdx.x == 0) sdone = P.st->done;
  fill_inv_mult(sinv);
  __syncthreads();
  if (sdone) return;
  const T alpha = (T)P.st->alpha;
  const T alpha_prev = XM == 2 ? (T)P.st->alpha_prev : T(0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // read by the next update, after this kernel
    if (XM == 1) {
      P.st->alpha_prev = P.st->alpha;
      P.st->xpend = 1;
    } else if (XM == 2) {
      P.st->xpend = 0;
    }
  }
  Acc rz, rr;
  const int64_t nv = P.n / W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t q = t0; q < nv; q += stride) {
    V pv, p2v, xv;
    if (XM != 1) {
      pv = reinterpret_cast<const V*>(P.p)[q];
      xv = reinterpret_cast<const V*>(P.x)[q];
    }
    if (XM == 2) p2v = reinterpret_cast<const V*>(P.p2)[q];
    const V wv = reinterpret_cast<const V*>(P.w)[q];
    V rv = reinterpret_cast<const V*>(P.r)[q];
    V mv;
    if (!EXT) mv = reinterpret_cast<const V*>(P.minv)[q];
    const M wm = reinterpret_cast<const M*>(P.wm)[q];
    V zv;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const T rq = VT::get(rv, k) - alpha * VT::get(wv, k);
      if (XM == 0) VT::set(xv, k, VT::get(xv, k) + alpha * VT::get(pv, k));
      if (XM == 2) VT::set(xv, k, (VT::get(xv, k) + alpha_prev * VT::get(p2v, k)) + alpha * VT::get(pv, k));
      VT::set(rv, k, rq);
      const T im = sinv[VT::getm(wm, k) & 0x7f];
      if (!EXT) {
        const T zq = VT::get(mv, k) * rq;
        VT::set(zv, k, zq);
        rz.add(rq * zq * im);
      }
      rr.add(rq * rq * im);
    }
    if (XM != 1) reinterpret_cast<V*>(P.x)[q] = xv;
    reinterpret_cast<V*>(P.r)[q] = rv;
    if (!EXT) reinterpret_cast<V*>(P.z)[q] = zv;
  }
  for (int64_t q = nv * W + t0; q < P.n; q += stride) {  // tail (n not a multiple of W)
    const T rq = P.r[q] - alpha * P.w[q];
    if (XM == 0) P.x[q] = P.x[q] + alpha * P.p[q];
    if (XM == 2) P.x[q] = (P.x[q] + alpha_prev * P.p2[q]) + alpha * P.p[q];
    P.r[q] = rq;
    const T im = sinv[P.wm[q] & 0x7f];
    if (!EXT) {
      const T zq = P.minv[q] * rq;
      P.z[q] = zq;
      rz.add(rq * zq * im);
    }
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
      } else if (st->delta2 > 0.0 && rr_t <= st->delta2 * st->rr_max) {
        st->done = 1;  // pause: the host replaces r by the FP64 true residual
        st->ru = 1;
      } else {
        if (rr_t > st->rr_max) st->rr_max = rr_t;
        if (!EXT) {
          st->beta = rz_t / st->rho;
          st->rho = rz_t;
        }
      }
      st->cnt[1] = 0;
    }
  }
}

// With an external preconditioner (z = M^{-1} r written by its kernels after
// k_pcg_update<T, true>): rho_new = <r, z>, beta = rho_new / rho_old.  If
// ZOUT, z is FP32 (computed from r scaled by zscale) and is written back to
// zout = z / zscale in T while the product is formed.
template <typename T, typename Z>
__global__ void __launch_bounds__(kVecThreads) k_pcg_rho(const T* __restrict__ r, const Z* __restrict__ z,
                                                         T* __restrict__ zout, double zscale, const uint8_t* wm,
                                                         int64_t n, PcgState* st, double* partial) {
  using Acc = typename AccOf<T>::type;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  __shared__ int sdone;
  if (threadIdx.x == 0) sdone = st->done;
  fill_inv_mult(sinv);
  __syncthreads();
  if (sdone) return;
  Acc rz;
  const T inv = (T)(1.0 / zscale);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    T zq = (T)z[q];
    if (zout) {
      zq = zq * inv;
      zout[q] = zq;
    }
    rz.add(r[q] * zq * sinv[wm[q] & 0x7f]);
  }
  const double a = block_sum(rz.get(), sred);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
  if (last_block(&st->cnt[3])) {
    const double rz_t = sum_partials(partial, gridDim.x, 1, 0, sred);
    if (threadIdx.x == 0) {
      if (rz_t != rz_t) {
        st->done = 1;
        st->status = 5;  // SEM_ERR_BREAKDOWN (NaN)
      } else {
        st->beta = rz_t / st->rho;
        st->rho = rz_t;
      }
      st->cnt[3] = 0;
    }
  }
}

// Start of a CG run on residual r (already b - A x0) and right-hand side b:
// z = M^{-1} r, p = 0, rho = <r,z>, rr = <r,r>, bb = <b,b>, beta = 0.
// EXT: z = M^{-1} r was written by the preconditioner's kernels (read here).
template <typename T, bool EXT>
__global__ void __launch_bounds__(kVecThreads) k_pcg_init(const VecParams<T> P) {
  using Acc = typename AccOf<T>::type;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  fill_inv_mult(sinv);
  __syncthreads();
  Acc rz, rr, bb;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.n; q += (int64_t)gridDim.x * blockDim.x) {
    const T rq = P.r[q], bq = P.b[q];
    T zq;
    if (EXT) {
      zq = P.z[q];
    } else {
      zq = P.minv[q] * rq;
      P.z[q] = zq;
    }
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
      st->rr_max = rr_t;
      st->ru = 0;
      st->cnt[2] = 0;
    }
  }
}

// Continue CG after the residual r was replaced (reliable update):
// z = M^{-1} r, rho_new = <r,z>, beta = rho_new / rho, rr_max = <r,r>; p is kept.
template <typename T, bool EXT>
__global__ void __launch_bounds__(kVecThreads) k_pcg_restart(const VecParams<T> P) {
  using Acc = typename AccOf<T>::type;
  __shared__ double sred[32];
  __shared__ T sinv[128];
  fill_inv_mult(sinv);
  __syncthreads();
  Acc rz, rr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.n; q += (int64_t)gridDim.x * blockDim.x) {
    const T rq = P.r[q];
    T zq;
    if (EXT) {
      zq = P.z[q];
    } else {
      zq = P.minv[q] * rq;
      P.z[q] = zq;
    }
    const T im = sinv[P.wm[q] & 0x7f];
    rz.add(rq * zq * im);
    rr.add(rq * rq * im);
  }
  const double a = block_sum(rz.get(), sred);
  const double b = block_sum(rr.get(), sred);
  if (threadIdx.x == 0) {
    P.partial[2 * blockIdx.x] = a;
    P.partial[2 * blockIdx.x + 1] = b;
  }
  if (last_block(&P.st->cnt[2])) {
    const double rz_t = sum_partials(P.partial, gridDim.x, 2, 0, sred);
    const double rr_t = sum_partials(P.partial, gridDim.x, 2, 1, sred);
    if (threadIdx.x == 0) {
      PcgState* st = P.st;
      st->beta = rz_t / st->rho;
      st->rho = rz_t;
      st->rr = rr_t;
      st->rr_max = rr_t;
      st->ru = 0;
      st->done = 0;
      st->status = 0;
      st->cnt[2] = 0;
    }
  }
}

template <typename T>
cudaError_t launch_pcg_restart(const VecParams<T>& p, cudaStream_t s, bool ext) {
  if (ext)
    k_pcg_restart<T, true><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else
    k_pcg_restart<T, false><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_pcg_restart<float>(const VecParams<float>&, cudaStream_t, bool);
template cudaError_t launch_pcg_restart<double>(const VecParams<double>&, cudaStream_t, bool);

template <typename T>
cudaError_t launch_pcg_update(const VecParams<T>& p, cudaStream_t s, bool ext, int xmode) {
  if (ext && xmode == 1)
    k_pcg_update<T, true, 1><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else if (ext && xmode == 2)
    k_pcg_update<T, true, 2><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else if (ext)
    k_pcg_update<T, true, 0><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else if (xmode == 1)
    k_pcg_update<T, false, 1><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else if (xmode == 2)
    k_pcg_update<T, false, 2><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else
    k_pcg_update<T, false, 0><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  return cudaGetLastError();
}

// A pair of x updates cut short by a pause (the first of the pair ran): x +=
// alpha_prev p2 and p = p2, so that x is current and the direction is back in
// p; nothing otherwise.  The caller clears xpend afterwards.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_pcg_xflush(T* __restrict__ x, T* __restrict__ p,
                                                           const T* __restrict__ p2, const PcgState* st, int64_t n) {
  if (!st->xpend) return;
  const T a = (T)st->alpha_prev;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const T v = p2[q];
    x[q] = x[q] + a * v;
    p[q] = v;
  }
}

template <typename T>
cudaError_t launch_pcg_xflush(T* x, T* p, const T* p2, PcgState* st, int64_t n, cudaStream_t s) {
  k_pcg_xflush<T><<<kVecBlocks, kVecThreads, 0, s>>>(x, p, p2, st, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&st->xpend, 0, sizeof(int), s);
}
template cudaError_t launch_pcg_xflush<float>(float*, float*, const float*, PcgState*, int64_t, cudaStream_t);
template cudaError_t launch_pcg_xflush<double>(double*, double*, const double*, PcgState*, int64_t, cudaStream_t);
template <typename T>
cudaError_t launch_pcg_init(const VecParams<T>& p, cudaStream_t s, bool ext) {
  if (ext)
    k_pcg_init<T, true><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  else
    k_pcg_init<T, false><<<kVecBlocks, kVecThreads, 0, s>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_pcg_update<double>(const VecParams<double>&, cudaStream_t, bool, int);
template cudaError_t launch_pcg_update<float>(const VecParams<float>&, cudaStream_t, bool, int);
template cudaError_t launch_pcg_init<double>(const VecParams<double>&, cudaStream_t, bool);
template cudaError_t launch_pcg_init<float>(const VecParams<float>&, cudaStream_t, bool);

template <typename T, typename Z>
cudaError_t launch_pcg_rho(const T* r, const Z* z, T* zout, double zscale, const uint8_t* wm, int64_t n, PcgState* st,
                           double* partial, cudaStream_t s) {
  k_pcg_rho<T, Z><<<kVecBlocks, kVecThreads, 0, s>>>(r, z, zout, zscale, wm, n, st, partial);
  return cudaGetLastError();
}
template cudaError_t launch_pcg_rho<double, double>(const double*, const double*, double*, double, const uint8_t*,
                                                    int64_t, PcgState*, double*, cudaStream_t);
template cudaError_t launch_pcg_rho<float, float>(const float*, const float*, float*, double, const uint8_t*, int64_t,
                                                  PcgState*, double*, cudaStream_t);
template cudaError_t launch_pcg_rho<double, float>(const double*, const float*, double*, double, const uint8_t*,
                                                   int64_t, PcgState*, double*, cudaStream_t);

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

__global__ void k_set_bb(PcgState* st, double bb, double delta2) {
  st->bb = bb;
  st->delta2 = delta2;
}
void launch_set_bb(PcgState* st, double bb, double delta2, cudaStream_t s) { k_set_bb<<<1, 1, 0, s>>>(st, bb, delta2); }

// pAp = fixed-order sum of a fused local operator's per-block partials; then
// alpha = rho / pAp, or a breakdown (one CTA, after the operator's launch)
__global__ void __launch_bounds__(1024) k_pap_finish(const double* __restrict__ partial, int count, PcgState* st) {
  __shared__ double sred[32];
  if (st->done) return;
  const double pAp = sum_partials(partial, count, 1, 0, sred);
  if (threadIdx.x == 0) {
    st->pAp = pAp;
    if (!(pAp > 0.0)) {
      st->done = 1;
      st->status = 5;  // SEM_ERR_BREAKDOWN
    } else {
      st->alpha = st->rho / pAp;
    }
  }
}
cudaError_t launch_pap_finish(const double* partial, int count, PcgState* st, cudaStream_t s) {
  k_pap_finish<<<1, 1024, 0, s>>>(partial, count, st);
  return cudaGetLastError();
}

__global__ void k_zero_f32(float* a, int64_t n) {
  GRID_STRIDE(q, n) a[q] = 0.f;
}
void launch_zero_f32(float* a, int64_t n, cudaStream_t s) { k_zero_f32<<<kVecBlocks, kVecThreads, 0, s>>>(a, n); }

}  // namespace sem
