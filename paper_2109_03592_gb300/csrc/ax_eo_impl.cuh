// FP64-accurate local operator (Alg. 1 + h2 mass term) in double-float
// arithmetic, even-odd form, for even n = N + 1.
//
// The GLL derivative matrix is centro-antisymmetric, D[n-1-i][n-1-l] =
// -D[i][l] (the nodes are symmetric about 0), and so is D^T.  For a pair of
// outputs (i, i' = n-1-i), i < n/2, of a contraction v -> D v:
//   P[l] = v[l] + v[l'],   M[l] = v[l] - v[l']              (l < n/2)
//   Ep[i][l] = (D[i][l] + D[i][l']) / 2,  Em[i][l] = (D[i][l] - D[i][l']) / 2
//   (D v)[i]  = sum_l Em[i][l] M[l] + sum_l Ep[i][l] P[l]
//   (D v)[i'] = sum_l Em[i][l] M[l] - sum_l Ep[i][l] P[l]
// so the two outputs cost n products instead of 2n.  In double-float a
// product term is ~12 FP32 instructions and a pre/post addition ~8, which
// makes the operator ~40% cheaper than the direct form (ax_df_impl.cuh).
//
// Thread mapping: one thread per 2x2x2 "octant" of an element, the points
// (i, j, k) with i in {a, n-1-a}, j in {b, n-1-b}, k in {c, n-1-c} for
// a, b, c < n/2, i.e. (n/2)^3 threads per element.  The pre-additions of all
// three directions and the post-additions are then inside one thread; the
// pre-added values go through shared memory, where the contractions of the
// other threads of the element read them.
//
// Values are kept as unnormalised pairs (s, c) with |c| of the order of the
// rounding errors of the magnitudes summed into s; such a pair enters the
// next product exactly like a normalised one, so the error stays ~2^-48 of
// the sum of the magnitudes of each contraction's terms.  h1 is folded into
// the forward coefficients (an FP64 product, split once per CTA).  u is split
// into its float pair from the bit pattern (split_bits), keeping the narrow
// FP64 pipe for the final hi + lo of w (measured 10% faster at N = 7 than
// FP64 conversions).  All float
// operations are explicit _rn intrinsics: the compiler may neither contract
// nor reorder them.
#pragma once

#include "ax_df_impl.cuh"

namespace sem {
namespace eo_detail {

using df_detail::DF;
using df_detail::join64;
using df_detail::mul_df;
using df_detail::split64;

struct Pair {
  float s, c;
};

// s + c = a * b (error-free product, cross terms of the low parts in c)
__device__ __forceinline__ Pair prod(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float c = __fmaf_rn(ah, bh, -p);
  c = __fmaf_rn(ah, bl, c);
  c = __fmaf_rn(al, bh, c);
  return Pair{p, c};
}

// A += a * b: the product's error and Knuth's TwoSum error go into A.c
__device__ __forceinline__ void madd(Pair& A, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float cc = __fadd_rn(A.c, pe);
  const float t = __fadd_rn(A.s, p);
  const float bp = __fsub_rn(t, A.s);
  const float e = __fadd_rn(__fsub_rn(A.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  A.s = t;
  A.c = __fadd_rn(cc, e);
}

// x = hi + lo from x's bit pattern with integer and FP32 operations only (the
// FP64 conversions of split64 run on GB300's narrow FP64 pipe): hi is x with
// its significand truncated to 24 bits, lo the remaining 29 bits rounded to
// nearest float, so |x - hi - lo| <= 2^-48 |x| for 2^-74 <= |x| < 2^128.
// Below 2^-74 lo is 0 and below 2^-126 hi is 0 too (entries that small do
// not change an FP64 result at the 1e-12 level unless the whole field is
// that small); |x| >= 2^128, infinities and NaNs give a NaN.
__device__ __forceinline__ Pair split_bits(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u, ah = hw & 0x7fffffffu;
  const unsigned hb = __funnelshift_l(lw, ah - (896u << 20), 3) | sign;  // float exponent + 23 significand bits
  float hi = ah >= (897u << 20) ? __uint_as_float(hb) : 0.f;
  hi = ah >= (1151u << 20) ? __uint_as_float(0x7fc00000u) : hi;
  // the 29 remaining significand bits as 23 + 6 exact floats, joined by one rounding
  const float r1 = __fsub_rn(__uint_as_float(0x4b000000u | ((lw >> 6) & 0x7fffffu)), 8388608.f);
  const float r0 = __fsub_rn(__uint_as_float(0x4b000000u | (lw & 0x3fu)), 8388608.f);
  const float r = __fmaf_rn(r1, 64.f, r0);
  const unsigned sb = (((ah - (948u << 20)) << 3) & 0x7f800000u) | sign;  // +-2^(E-1075), E the biased exponent
  const float lo = ah >= (949u << 20) ? __fmul_rn(r, __uint_as_float(sb)) : 0.f;
  return Pair{hi, lo};
}

// a + b and a - b (TwoSum on the high parts)
__device__ __forceinline__ Pair add(Pair a, Pair b) {
  const float t = __fadd_rn(a.s, b.s);
  const float bp = __fsub_rn(t, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b.s, bp));
  return Pair{t, __fadd_rn(e, __fadd_rn(a.c, b.c))};
}
__device__ __forceinline__ Pair sub(Pair a, Pair b) { return add(a, Pair{-b.s, -b.c}); }

// Shared-memory index of point (i, j, k) in one element's array of float2.
// n = 8: XOR swizzle of i by (j, k) -- every access pattern of the kernel
// (octant stores; r, s and t reads) is free of bank conflicts.  Other n:
// padded rows and planes chosen by the same conflict count.
template <int n>
struct EoLayout {
  static constexpr int RP = n == 6 ? 11 : n == 10 ? 11 : n == 12 ? 13 : n;
  static constexpr int PL = n == 6 ? 68 : n == 10 ? 119 : n == 12 ? 168 : n * n;
  static constexpr int size = n * PL;
  __device__ static __forceinline__ int idx(int i, int j, int k) { return i + RP * j + PL * k; }
};
template <>
struct EoLayout<8> {
  static constexpr int size = 512;
  __device__ static __forceinline__ int idx(int i, int j, int k) {
    const int sw = 4 * (((j >> 1) ^ k) & 1) + 2 * (k & 1);
    return (i ^ sw) + 8 * j + 64 * k;
  }
};

constexpr int eo_threads_per_element_v(int N) { return ((N + 1) / 2) * ((N + 1) / 2) * ((N + 1) / 2); }
template <int N>
constexpr int eo_threads_per_element() {
  return eo_threads_per_element_v(N);
}

// Register budget: 640 resident threads per SM (96 registers at 128 threads
// per CTA, 128 at 256) measured fastest at N = 7 and 11.
constexpr int eo_min_blocks(int threads) { return 640 / threads < 1 ? 1 : 640 / threads; }

template <int N, int EPB, bool FUSED>
__global__ void __launch_bounds__(EPB* eo_threads_per_element<N>(), eo_min_blocks(EPB* eo_threads_per_element<N>()))
    k_ax_eo(const AxDFParams P) {
  static_assert((N & 1) == 1, "even-odd kernel needs an even number of points per direction");
  constexpr int n = N + 1, h = n / 2, T = h * h * h, n2 = n * n, n3 = n2 * n;
  using L = EoLayout<n>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sC = reinterpret_cast<float4*>(smem_raw);  // [2][h][h]: (Ep.hi, Ep.lo, Em.hi, Em.lo), fwd then bwd
  float2* sA = reinterpret_cast<float2*>(sC + 2 * h * h);
  __shared__ double sred[32];
  __shared__ int sdone;

  const int tid = threadIdx.x;
  if (FUSED) {
    if (tid == 0) sdone = P.st->done;
    __syncthreads();
    if (sdone) return;
  }
  // The CTA's G (hi and lo) into L2 while the forward contractions run: one
  // bulk prefetch per array (a hint, nothing waits on it), so the G loads of
  // the pointwise step hit L2 instead of waiting on DRAM.
  if (tid == 0) {
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int64_t ne = min((int64_t)EPB, P.E - e0);
    const uint32_t bytes = (uint32_t)(ne * 6 * n3 * sizeof(float));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.Ghi + e0 * 6 * n3), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.Glo + e0 * 6 * n3), "r"(bytes) : "memory");
  }
  // coefficient tables; h1 scales the forward ones
  if (P.h1 == 1.0) {
    for (int q = tid; q < 2 * h * h; q += blockDim.x) sC[q] = reinterpret_cast<const float4*>(P.eodf)[q];
  } else {
    for (int q = tid; q < 2 * h * h; q += blockDim.x) {
      const double sc = q < h * h ? P.h1 : 1.0;
      const DF ep = split64(sc * P.eo64[2 * q]), em = split64(sc * P.eo64[2 * q + 1]);
      sC[q] = make_float4(ep.h, ep.l, em.h, em.l);
    }
  }

  const int le = tid / T, t = tid - le * T;
  const int a = t % h, b = (t / h) % h, c = t / (h * h);
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool act = e < P.E;
  float2* S0 = sA + (size_t)le * 3 * L::size;
  float2* S1 = S0 + L::size;
  float2* S2 = S1 + L::size;
  const int I[2] = {a, n - 1 - a}, J[2] = {b, n - 1 - b}, K[2] = {c, n - 1 - c};
  // octant point q = da + 2 db + 4 dc is (I[da], J[db], K[dc])
  const int64_t base = e * n3;

  // u - u0 with u0 the value at the element's first point: the stiffness part
  // annihilates constants, and without the shift a smooth field with a large
  // mean loses its low-order bits in the contractions (measured 2e-12 instead
  // of 2e-13 against the FP64 oracle).  The mass term and <p, A_L p> add u0 back.
  Pair u[8];
  double u0 = 0.0, beta = 0.0;
  if (act) {
    if (FUSED) {
      beta = P.st->beta;
      u0 = P.z[base] + beta * P.p[base];
    } else {
      u0 = P.u[base];
    }
  }
  // every thread has read p at the element's first point before its owner overwrites it
  if (FUSED) __syncthreads();
  if (act) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t g = base + I[q & 1] + n * J[(q >> 1) & 1] + n2 * K[q >> 2];
      double v;
      if (FUSED) {
        v = P.z[g] + beta * P.p[g];
        (P.pout ? P.pout : P.p)[g] = v;
      } else {
        v = P.u[g];
      }
      u[q] = split_bits(v - u0);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) u[q] = Pair{0.f, 0.f};
  }

  // pre-additions of the three directions; P at the pair's low index, M at its high one
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      {  // r: pairs over da, row (db, dc) = (x, y)
        const Pair p = add(u[2 * x + 4 * y], u[1 + 2 * x + 4 * y]), m = sub(u[2 * x + 4 * y], u[1 + 2 * x + 4 * y]);
        S0[L::idx(a, J[x], K[y])] = make_float2(p.s, p.c);
        S0[L::idx(n - 1 - a, J[x], K[y])] = make_float2(m.s, m.c);
      }
      {  // s: pairs over db, row (da, dc) = (x, y)
        const Pair p = add(u[x + 4 * y], u[x + 2 + 4 * y]), m = sub(u[x + 4 * y], u[x + 2 + 4 * y]);
        S1[L::idx(I[x], b, K[y])] = make_float2(p.s, p.c);
        S1[L::idx(I[x], n - 1 - b, K[y])] = make_float2(m.s, m.c);
      }
      {  // t: pairs over dc, row (da, db) = (x, y)
        const Pair p = add(u[x + 2 * y], u[x + 2 * y + 4]), m = sub(u[x + 2 * y], u[x + 2 * y + 4]);
        S2[L::idx(I[x], J[y], c)] = make_float2(p.s, p.c);
        S2[L::idx(I[x], J[y], n - 1 - c)] = make_float2(m.s, m.c);
      }
    }
  __syncthreads();

  // forward contractions: g[d][q] = (h1 D_d u)(point q), d = r, s, t
  Pair g[3][8];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float4 cf[h];
    const int own = d == 0 ? a : d == 1 ? b : c;
#pragma unroll
    for (int l = 0; l < h; ++l) cf[l] = sC[own * h + l];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        Pair Ap, Bm;
#pragma unroll
        for (int l = 0; l < h; ++l) {
          float2 pv, mv;
          if (d == 0) {
            pv = S0[L::idx(l, J[x], K[y])];
            mv = S0[L::idx(n - 1 - l, J[x], K[y])];
          } else if (d == 1) {
            pv = S1[L::idx(I[x], l, K[y])];
            mv = S1[L::idx(I[x], n - 1 - l, K[y])];
          } else {
            pv = S2[L::idx(I[x], J[y], l)];
            mv = S2[L::idx(I[x], J[y], n - 1 - l)];
          }
          if (l == 0) {
            Ap = prod(cf[0].x, cf[0].y, pv.x, pv.y);
            Bm = prod(cf[0].z, cf[0].w, mv.x, mv.y);
          } else {
            madd(Ap, cf[l].x, cf[l].y, pv.x, pv.y);
            madd(Bm, cf[l].z, cf[l].w, mv.x, mv.y);
          }
        }
        // the pair's low point gets Bm + Ap, its high point Bm - Ap
        const int q0 = d == 0 ? 2 * x + 4 * y : d == 1 ? x + 4 * y : x + 2 * y;
        const int q1 = q0 + (d == 0 ? 1 : d == 1 ? 2 : 4);
        g[d][q0] = add(Bm, Ap);
        g[d][q1] = sub(Bm, Ap);
      }
  }

  // (wr, ws, wt) = G (ur, us, ut); g1..g6 = G_rr, G_ss, G_tt, G_rs, G_rt, G_st
  if (act) {
    const float* Gh = P.Ghi + e * 6 * n3;
    const float* Gl = P.Glo + e * 6 * n3;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int off = I[q & 1] + n * J[(q >> 1) & 1] + n2 * K[q >> 2];
      float gh[6], gl[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        gh[f] = Gh[f * n3 + off];
        gl[f] = Gl[f * n3 + off];
      }
      const Pair ur = g[0][q], us = g[1][q], ut = g[2][q];
      Pair wr = prod(gh[0], gl[0], ur.s, ur.c);
      madd(wr, gh[3], gl[3], us.s, us.c);
      madd(wr, gh[4], gl[4], ut.s, ut.c);
      Pair ws = prod(gh[3], gl[3], ur.s, ur.c);
      madd(ws, gh[1], gl[1], us.s, us.c);
      madd(ws, gh[5], gl[5], ut.s, ut.c);
      Pair wt = prod(gh[4], gl[4], ur.s, ur.c);
      madd(wt, gh[5], gl[5], us.s, us.c);
      madd(wt, gh[2], gl[2], ut.s, ut.c);
      g[0][q] = wr;
      g[1][q] = ws;
      g[2][q] = wt;
    }
  }
  __syncthreads();  // every forward read of S0..S2 is done

#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      {
        const Pair p = add(g[0][2 * x + 4 * y], g[0][1 + 2 * x + 4 * y]);
        const Pair m = sub(g[0][2 * x + 4 * y], g[0][1 + 2 * x + 4 * y]);
        S0[L::idx(a, J[x], K[y])] = make_float2(p.s, p.c);
        S0[L::idx(n - 1 - a, J[x], K[y])] = make_float2(m.s, m.c);
      }
      {
        const Pair p = add(g[1][x + 4 * y], g[1][x + 2 + 4 * y]), m = sub(g[1][x + 4 * y], g[1][x + 2 + 4 * y]);
        S1[L::idx(I[x], b, K[y])] = make_float2(p.s, p.c);
        S1[L::idx(I[x], n - 1 - b, K[y])] = make_float2(m.s, m.c);
      }
      {
        const Pair p = add(g[2][x + 2 * y], g[2][x + 2 * y + 4]), m = sub(g[2][x + 2 * y], g[2][x + 2 * y + 4]);
        S2[L::idx(I[x], J[y], c)] = make_float2(p.s, p.c);
        S2[L::idx(I[x], J[y], n - 1 - c)] = make_float2(m.s, m.c);
      }
    }
  __syncthreads();

  // back contractions with D^T: w(point) = sum over d of (D_d^T w_d)(point)
  Pair o[8];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float4 cf[h];
    const int own = d == 0 ? a : d == 1 ? b : c;
#pragma unroll
    for (int l = 0; l < h; ++l) cf[l] = sC[h * h + own * h + l];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        Pair Ap, Bm;
#pragma unroll
        for (int l = 0; l < h; ++l) {
          float2 pv, mv;
          if (d == 0) {
            pv = S0[L::idx(l, J[x], K[y])];
            mv = S0[L::idx(n - 1 - l, J[x], K[y])];
          } else if (d == 1) {
            pv = S1[L::idx(I[x], l, K[y])];
            mv = S1[L::idx(I[x], n - 1 - l, K[y])];
          } else {
            pv = S2[L::idx(I[x], J[y], l)];
            mv = S2[L::idx(I[x], J[y], n - 1 - l)];
          }
          if (l == 0) {
            Ap = prod(cf[0].x, cf[0].y, pv.x, pv.y);
            Bm = prod(cf[0].z, cf[0].w, mv.x, mv.y);
          } else {
            madd(Ap, cf[l].x, cf[l].y, pv.x, pv.y);
            madd(Bm, cf[l].z, cf[l].w, mv.x, mv.y);
          }
        }
        const int q0 = d == 0 ? 2 * x + 4 * y : d == 1 ? x + 4 * y : x + 2 * y;
        const int q1 = q0 + (d == 0 ? 1 : d == 1 ? 2 : 4);
        if (d == 0) {
          o[q0] = add(Bm, Ap);
          o[q1] = sub(Bm, Ap);
        } else {
          o[q0] = add(o[q0], add(Bm, Ap));
          o[q1] = add(o[q1], sub(Bm, Ap));
        }
      }
  }

  Pair pw{0.f, 0.f};  // this thread's part of <p, A_L p> = <p - u0, w> + u0 * sum(w)
  Pair sw{0.f, 0.f};
  if (act) {
    const DF h2 = split64(P.h2);
    const Pair c0 = split_bits(FUSED ? (P.pout ? P.pout : P.p)[base] : P.u[base]);  // u0 again (not kept live in registers)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t gi = base + I[q & 1] + n * J[(q >> 1) & 1] + n2 * K[q >> 2];
      Pair r = o[q];
      if (P.helm) {  // + h2 B (u - u0) + h2 B u0, B = Bhi + Blo
        const DF hb = mul_df(h2, DF{P.Bhi[gi], P.Blo[gi]});
        r = add(r, prod(hb.h, hb.l, u[q].s, u[q].c));
        r = add(r, prod(hb.h, hb.l, c0.s, c0.c));
      }
      P.w[gi] = join64(DF{r.s, r.c});
      if (FUSED) {
        madd(pw, u[q].s, u[q].c, r.s, r.c);
        sw = add(sw, r);
      }
    }
    if (FUSED) madd(pw, c0.s, c0.c, sw.s, sw.c);
  }

  if (FUSED) {  // this block's part of <p, A_L p>; k_pap_finish sums the parts in block order
    const double s = block_sum((double)pw.s + (double)pw.c, sred);
    if (tid == 0) P.partial[blockIdx.x] = s;
  }
}

template <int N, int EPB, bool FUSED>
cudaError_t launch_eo_t(const AxDFParams& p, cudaStream_t s, int* grid_out) {
  constexpr int n = N + 1, h = n / 2;
  const size_t smem = sizeof(float4) * 2 * h * h + sizeof(float2) * 3ull * EPB * EoLayout<n>::size;
  static DeviceOnce once;
  cudaError_t aerr = once.get([&](int, int*) {
    return cudaFuncSetAttribute(k_ax_eo<N, EPB, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (aerr != cudaSuccess) return aerr;
  if (!p.eo64 || !p.eodf) return cudaErrorInvalidValue;
  const int64_t grid = (p.E + EPB - 1) / EPB;
  if (grid_out) *grid_out = (int)grid;
  if (p.E == 0) return cudaSuccess;
  k_ax_eo<N, EPB, FUSED><<<(unsigned)grid, EPB * eo_threads_per_element<N>(), smem, s>>>(p);
  cudaError_t err = cudaGetLastError();
  // a separate one-CTA sum of the block partials: the operator's 1e4-1e5
  // blocks then need no grid-wide arrival counter (fence + atomic per block)
  if (FUSED && err == cudaSuccess) err = launch_pap_finish(p.partial, (int)grid, p.st, s);
  return err;
}

constexpr int epb_eo(int N, int variant) {
  return (variant == 2 ? 128 : 256) / eo_threads_per_element_v(N) < 1
             ? 1
             : (variant == 2 ? 128 : 256) / eo_threads_per_element_v(N);
}

}  // namespace eo_detail

// FP64-accurate (double-float) local operator of order N: variants 0 and 1
// are the direct kernels (ax_df_impl.cuh), 2 and 3 the even-odd kernels with
// ~128 / ~256 threads per CTA (odd N only).
template <int N>
inline cudaError_t dispatch_fp64df_n(int variant, bool fused, const AxDFParams& p, cudaStream_t s, int* grid_out) {
  using namespace eo_detail;
  if (variant < 2) return df_detail::dispatch_df_n<N>(variant, fused, p, s, grid_out);
  if constexpr ((N & 1) == 1) {
    if (variant == 2)
      return fused ? launch_eo_t<N, epb_eo(N, 2), true>(p, s, grid_out)
                   : launch_eo_t<N, epb_eo(N, 2), false>(p, s, grid_out);
    if (variant == 3)
      return fused ? launch_eo_t<N, epb_eo(N, 3), true>(p, s, grid_out)
                   : launch_eo_t<N, epb_eo(N, 3), false>(p, s, grid_out);
  }
  return cudaErrorNotSupported;
}

}  // namespace sem
