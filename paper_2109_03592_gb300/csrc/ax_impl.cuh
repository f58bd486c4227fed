// The matrix-free local SEM operator of Alg. 1 (CUDA Fortran `axhelm`),
// re-designed for sm_103a.
//
// Per element and GLL point (i,j,k), Alg. 1 computes
//   ur = sum_l D_il u_ljk,  us = sum_l D_jl u_ilk,  ut = sum_l D_kl u_ijl
//   (wr, ws, wt) = h1 G (ur, us, ut),  G = [[g1,g4,g5],[g4,g2,g6],[g5,g6,g3]]
//   w_ijk = sum_l D_li wr_ljk + D_lj ws_ilk + D_lk wt_ijl
// and the Helmholtz problem of Sec. 2, Eq. 4 adds h2 B_ijk u_ijk.
//
// Thread mapping (differs from the listing's one thread per point): a thread
// owns one (i,j) column of an element and walks k.  The column of u stays in
// registers, so the t-contraction and the D^T_t back-contraction never touch
// shared memory; only the r and s directions go through shared memory (three
// n^3 arrays per element, rows padded to n+1 to keep the FP64 accesses free
// of bank conflicts).  h1 is a scalar, so it is applied once to the sum of the
// back-contractions instead of to wr, ws, wt.
#pragma once

#include <type_traits>

#include "ax_tma.cuh"
#include "kernels.h"

namespace sem {

template <int N, typename T, int EPB, bool FUSED>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1)) k_ax(const AxParams<T> P) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  constexpr int RP = n + 1, PL = n * RP;  // padded row / plane strides in shared memory
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);  // D[a][b] at a*RP + b
  T* su = sD + n * RP;
  T* swr = su + EPB * n * PL;
  T* sws = swr + EPB * n * PL;
  __shared__ double sred[32];
  __shared__ int sdone;

  const int tid = threadIdx.x;
  if (FUSED) {
    if (tid == 0) sdone = P.st->done;
    __syncthreads();
    if (sdone) return;
  }
  for (int q = tid; q < n2; q += blockDim.x) sD[(q / n) * RP + (q % n)] = P.D[q];

  const int le = tid / n2, ij = tid - le * n2, i = ij % n, j = ij / n;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool act = e < P.E;
  T* sue = su + le * n * PL;
  T* swre = swr + le * n * PL;
  T* swse = sws + le * n * PL;
  const int64_t base = e * n3 + ij;

  T ru[n];
  if (act) {
    if (FUSED) {
      const T beta = (T)P.st->beta;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const T v = P.z[base + k * n2] + beta * P.p[base + k * n2];
        (P.pout ? P.pout : P.p)[base + k * n2] = v;
        ru[k] = v;
      }
    } else {
#pragma unroll
      for (int k = 0; k < n; ++k) ru[k] = P.u[base + k * n2];
    }
#pragma unroll
    for (int k = 0; k < n; ++k) sue[k * PL + j * RP + i] = ru[k];
  }
  __syncthreads();

  T rw[n];
#pragma unroll
  for (int k = 0; k < n; ++k) rw[k] = T(0);
  if (act) {
    const T* Ge = P.G + e * 6 * n3 + ij;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const T g1 = Ge[k * n2], g2 = Ge[n3 + k * n2], g3 = Ge[2 * n3 + k * n2];
      const T g4 = Ge[3 * n3 + k * n2], g5 = Ge[4 * n3 + k * n2], g6 = Ge[5 * n3 + k * n2];
      T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        ur += sD[i * RP + l] * sue[k * PL + j * RP + l];
        us += sD[j * RP + l] * sue[k * PL + l * RP + i];
        ut += sD[k * RP + l] * ru[l];
      }
      const T wr = g1 * ur + g4 * us + g5 * ut;
      const T ws = g4 * ur + g2 * us + g6 * ut;
      const T wt = g5 * ur + g6 * us + g3 * ut;
      swre[k * PL + j * RP + i] = wr;
      swse[k * PL + j * RP + i] = ws;
#pragma unroll
      for (int k2 = 0; k2 < n; ++k2) rw[k2] += sD[k * RP + k2] * wt;
    }
  }
  __syncthreads();

  T pw = T(0);  // this thread's part of <p, A_L p> (n terms, accumulated in T)
  if (act) {
    // the n values of B first, all in flight together: loaded next to the
    // stores of w, each load waited in turn (w and B may alias for the compiler)
    T rb[n];
#pragma unroll
    for (int k = 0; k < n; ++k) rb[k] = P.helm ? __ldg(P.B + base + k * n2) : T(0);
#pragma unroll
    for (int k = 0; k < n; ++k) {
      T acc = rw[k];
#pragma unroll
      for (int l = 0; l < n; ++l)
        acc += sD[l * RP + i] * swre[k * PL + j * RP + l] + sD[l * RP + j] * swse[k * PL + l * RP + i];
      T out = P.h1 * acc;
      if (P.helm) out += P.h2 * rb[k] * ru[k];
      P.w[base + k * n2] = out;
      if (FUSED) pw += ru[k] * out;
    }
  }

  if (FUSED) {  // this block's part of <p, A_L p>; k_pap_finish sums the parts in block order
    const double s = block_sum((double)pw, sred);
    if (tid == 0) P.partial[blockIdx.x] = s;
  }
}

template <int N, typename T, int EPB>
size_t ax_smem_bytes() {
  constexpr int n = N + 1;
  return sizeof(T) * ((size_t)n * (n + 1) + 3ull * EPB * n * n * (n + 1));
}

template <int N, typename T, int EPB, bool FUSED>
cudaError_t launch_ax_t(const AxParams<T>& p, cudaStream_t s, int* grid_out) {
  constexpr int n = N + 1;
  const size_t smem = ax_smem_bytes<N, T, EPB>();
  static DeviceOnce once;
  cudaError_t aerr = once.get([&](int, int*) {
    return cudaFuncSetAttribute(k_ax<N, T, EPB, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (aerr != cudaSuccess) return aerr;
  const int64_t grid = (p.E + EPB - 1) / EPB;
  if (grid_out) *grid_out = (int)grid;
  if (p.E == 0) return cudaSuccess;
  k_ax<N, T, EPB, FUSED><<<(unsigned)grid, EPB * n * n, smem, s>>>(p);
  cudaError_t err = cudaGetLastError();
  if (FUSED && err == cudaSuccess) err = launch_pap_finish(p.partial, (int)grid, p.st, s);
  return err;
}

// Elements per block: about 256 threads (variant 0) or about 128 (variant 1).
constexpr int epb_for(int N, int variant) {
  return ((variant == 0 ? 256 : 128) / ((N + 1) * (N + 1))) < 1 ? 1
                                                                   : ((variant == 0 ? 256 : 128) / ((N + 1) * (N + 1)));
}

template <typename T, int N>
cudaError_t dispatch_ax_n(int variant, bool fused, const AxParams<T>& p, cudaStream_t s, int* grid_out) {
  if (variant >= 2) {
    if constexpr (std::is_same<T, float>::value && (N % 2 == 1)) {
      if (variant == 2)
        return fused ? tma::launch_ax_tma_t<N, epb_for(N, 1), 3, true>(p, p.err, s, grid_out)
                     : tma::launch_ax_tma_t<N, epb_for(N, 1), 3, false>(p, p.err, s, grid_out);
      if (variant == 3)
        return fused ? tma::launch_ax_tma_t<N, epb_for(N, 0), 2, true>(p, p.err, s, grid_out)
                     : tma::launch_ax_tma_t<N, epb_for(N, 0), 2, false>(p, p.err, s, grid_out);
    }
    return cudaErrorNotSupported;
  }
  if (variant == 0) {
    return fused ? launch_ax_t<N, T, epb_for(N, 0), true>(p, s, grid_out)
                 : launch_ax_t<N, T, epb_for(N, 0), false>(p, s, grid_out);
  }
  return fused ? launch_ax_t<N, T, epb_for(N, 1), true>(p, s, grid_out)
               : launch_ax_t<N, T, epb_for(N, 1), false>(p, s, grid_out);
}

}  // namespace sem
