// FP64-accurate local operator (Alg. 1 + h2 mass term) computed in
// double-float arithmetic on the FP32 pipe.
//
// GB300 issues FP64 FMAs at ~1/60 of its FP32 rate, so the native FP64
// kernel (ax_impl.cuh) is bound by the FP64 pipe long before HBM.  Here every
// value of the contraction is an unevaluated pair (hi, lo) of floats with
// |lo| <= ulp(hi)/2 (about 48 significant bits):
//   * D = Dhi + Dlo and G = Ghi + Glo are split once at mesh set-up;
//   * u (FP64 in memory) is split on load, w is rounded back to FP64 on store;
//   * each term a*b of a contraction is formed exactly as p + e with
//     p = fl(ahi*bhi), e = fma(ahi, bhi, -p) + ahi*blo + alo*bhi
//     (Dekker/Knuth error-free product via FMA), the running sum of the p's is
//     kept error-free with Knuth's TwoSum, and all error terms are summed in
//     plain FP32 (they are ~2^-24 of the terms, so that sum is good to
//     ~2^-48 of them);
//   * the pair is renormalised once per output (Fast2Sum).
// The result agrees with an FP64 evaluation to ~1e-14 relative, inside the
// 1e-12 bound required of the FP64 operator.
// All float operations use explicit _rn intrinsics so that the compiler
// cannot contract or reorder them.
#pragma once

#include "kernels.h"

namespace sem {
namespace df_detail {


struct DF {
  float h, l;
};

__device__ __forceinline__ DF split64(double x) {
  const float h = __double2float_rn(x);
  return DF{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double join64(DF a) { return (double)a.h + (double)a.l; }

// Product of two double-float numbers (Dekker), renormalised.
__device__ __forceinline__ DF mul_df(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float t = __fadd_rn(p, e);
  return DF{t, __fsub_rn(e, __fsub_rn(t, p))};
}

// Lazily-compensated dot-product accumulator.
struct Acc {
  float s, c;
  __device__ __forceinline__ void zero() {
    s = 0.f;
    c = 0.f;
  }
  // += a * b
  __device__ __forceinline__ void madd(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float pe = __fmaf_rn(ah, bh, -p);
    pe = __fmaf_rn(ah, bl, pe);
    pe = __fmaf_rn(al, bh, pe);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ DF result() const {
    const float t = __fadd_rn(s, c);
    return DF{t, __fsub_rn(c, __fsub_rn(t, s))};
  }
};

template <int N, int EPB, bool FUSED>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1)) k_ax_df(const AxDFParams P) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  constexpr int RP = n + 1, PL = n * RP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sD = reinterpret_cast<float2*>(smem_raw);  // (Dhi, Dlo) at a*RP + b
  float2* su = sD + n * RP;
  float2* swr = su + EPB * n * PL;
  float2* sws = swr + EPB * n * PL;
  __shared__ double sred[32];
  __shared__ int sdone;

  const int tid = threadIdx.x;
  if (FUSED) {
    if (tid == 0) sdone = P.st->done;
    __syncthreads();
    if (sdone) return;
  }
  for (int q = tid; q < n2; q += blockDim.x) sD[(q / n) * RP + (q % n)] = make_float2(P.Dhi[q], P.Dlo[q]);

  const int le = tid / n2, ij = tid - le * n2, i = ij % n, j = ij / n;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool act = e < P.E;
  float2* sue = su + le * n * PL;
  float2* swre = swr + le * n * PL;
  float2* swse = sws + le * n * PL;
  const int64_t base = e * n3 + ij;

  // u - u0 with u0 the value at the element's first point: the stiffness part
  // annihilates constants, and the shift keeps a smooth field's large mean out
  // of the contractions' rounding; the mass term and <p, A_L p> add u0 back.
  double ud[n];
  DF ru[n];
  double u0 = 0.0, beta = 0.0;
  if (act && FUSED) {
    beta = P.st->beta;
    u0 = P.z[e * n3] + beta * P.p[e * n3];
  }
  // every thread has read p at the element's first point before its owner overwrites it
  if (FUSED) __syncthreads();
  if (act) {
    if (FUSED) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const double v = P.z[base + k * n2] + beta * P.p[base + k * n2];
        (P.pout ? P.pout : P.p)[base + k * n2] = v;
        ud[k] = v;
      }
    } else {
      u0 = P.u[e * n3];
#pragma unroll
      for (int k = 0; k < n; ++k) ud[k] = P.u[base + k * n2];
    }
#pragma unroll
    for (int k = 0; k < n; ++k) {
      ru[k] = split64(ud[k] - u0);
      sue[k * PL + j * RP + i] = make_float2(ru[k].h, ru[k].l);
    }
  }
  __syncthreads();

  Acc rw[n];
#pragma unroll
  for (int k = 0; k < n; ++k) rw[k].zero();
  if (act) {
    const float* Gh = P.Ghi + e * 6 * n3 + ij;
    const float* Gl = P.Glo + e * 6 * n3 + ij;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      float gh[6], gl[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        gh[c] = Gh[c * n3 + k * n2];
        gl[c] = Gl[c * n3 + k * n2];
      }
      Acc ar, as, at;
      ar.zero();
      as.zero();
      at.zero();
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const float2 di = sD[i * RP + l], dj = sD[j * RP + l], dk = sD[k * RP + l];
        const float2 a = sue[k * PL + j * RP + l], b = sue[k * PL + l * RP + i];
        ar.madd(di.x, di.y, a.x, a.y);
        as.madd(dj.x, dj.y, b.x, b.y);
        at.madd(dk.x, dk.y, ru[l].h, ru[l].l);
      }
      const DF ur = ar.result(), us = as.result(), ut = at.result();
      Acc xr, xs, xt;
      xr.zero();
      xs.zero();
      xt.zero();
      // (wr, ws, wt) = G (ur, us, ut); g1..g6 = G_rr, G_ss, G_tt, G_rs, G_rt, G_st
      xr.madd(gh[0], gl[0], ur.h, ur.l);
      xr.madd(gh[3], gl[3], us.h, us.l);
      xr.madd(gh[4], gl[4], ut.h, ut.l);
      xs.madd(gh[3], gl[3], ur.h, ur.l);
      xs.madd(gh[1], gl[1], us.h, us.l);
      xs.madd(gh[5], gl[5], ut.h, ut.l);
      xt.madd(gh[4], gl[4], ur.h, ur.l);
      xt.madd(gh[5], gl[5], us.h, us.l);
      xt.madd(gh[2], gl[2], ut.h, ut.l);
      const DF wr = xr.result(), ws = xs.result(), wt = xt.result();
      swre[k * PL + j * RP + i] = make_float2(wr.h, wr.l);
      swse[k * PL + j * RP + i] = make_float2(ws.h, ws.l);
#pragma unroll
      for (int k2 = 0; k2 < n; ++k2) {
        const float2 d = sD[k * RP + k2];
        rw[k2].madd(d.x, d.y, wt.h, wt.l);
      }
    }
  }
  __syncthreads();

  Acc pw;  // this thread's part of <p, A_L p>, in double-float
  pw.zero();
  if (act) {
    const DF h1 = split64(P.h1);
    const DF h2 = split64(P.h2);
    const DF c0 = split64(FUSED ? (P.pout ? P.pout : P.p)[e * n3] : P.u[e * n3]);  // u0 again (not kept live in registers)
#pragma unroll
    for (int k = 0; k < n; ++k) {
      Acc acc = rw[k];
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const float2 di = sD[l * RP + i], dj = sD[l * RP + j];
        const float2 a = swre[k * PL + j * RP + l], b = swse[k * PL + l * RP + i];
        acc.madd(di.x, di.y, a.x, a.y);
        acc.madd(dj.x, dj.y, b.x, b.y);
      }
      const DF s = acc.result();
      Acc sc;
      sc.zero();
      sc.madd(h1.h, h1.l, s.h, s.l);
      if (P.helm) {
        // + h2 B (u - u0) + h2 B u0, with B = Bhi + Blo
        const DF hb = mul_df(h2, DF{P.Bhi[base + k * n2], P.Blo[base + k * n2]});
        sc.madd(hb.h, hb.l, ru[k].h, ru[k].l);
        sc.madd(hb.h, hb.l, c0.h, c0.l);
      }
      const DF o = sc.result();
      P.w[base + k * n2] = join64(o);
      if (FUSED) {
        pw.madd(ru[k].h, ru[k].l, o.h, o.l);
        pw.madd(c0.h, c0.l, o.h, o.l);
      }
    }
  }

  if (FUSED) {  // this block's part of <p, A_L p>; k_pap_finish sums the parts in block order
    const DF pr = pw.result();
    const double s = block_sum((double)pr.h + (double)pr.l, sred);
    if (tid == 0) P.partial[blockIdx.x] = s;
  }
}

template <int N, int EPB, bool FUSED>
cudaError_t launch_df_t(const AxDFParams& p, cudaStream_t s, int* grid_out) {
  constexpr int n = N + 1;
  const size_t smem = sizeof(float2) * ((size_t)n * (n + 1) + 3ull * EPB * n * n * (n + 1));
  static DeviceOnce once;
  cudaError_t aerr = once.get([&](int, int*) {
    return cudaFuncSetAttribute(k_ax_df<N, EPB, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (aerr != cudaSuccess) return aerr;
  const int64_t grid = (p.E + EPB - 1) / EPB;
  if (grid_out) *grid_out = (int)grid;
  if (p.E == 0) return cudaSuccess;
  k_ax_df<N, EPB, FUSED><<<(unsigned)grid, EPB * n * n, smem, s>>>(p);
  cudaError_t err = cudaGetLastError();
  if (FUSED && err == cudaSuccess) err = launch_pap_finish(p.partial, (int)grid, p.st, s);
  return err;
}

constexpr int epb_df(int N, int variant) {
  return ((variant == 0 ? 256 : 128) / ((N + 1) * (N + 1))) < 1 ? 1
                                                                   : ((variant == 0 ? 256 : 128) / ((N + 1) * (N + 1)));
}

template <int N>
inline cudaError_t dispatch_df_n(int variant, bool fused, const AxDFParams& p, cudaStream_t s, int* grid_out) {
  if (variant >= 2) return cudaErrorNotSupported;
  if (variant == 0)
    return fused ? launch_df_t<N, epb_df(N, 0), true>(p, s, grid_out)
                 : launch_df_t<N, epb_df(N, 0), false>(p, s, grid_out);
  return fused ? launch_df_t<N, epb_df(N, 1), true>(p, s, grid_out)
               : launch_df_t<N, epb_df(N, 1), false>(p, s, grid_out);
}

}  // namespace df_detail
}  // namespace sem
