// Line-based sum factorisation of the pressure operator's weak divergence
// and gradient (included by pressure.cu; the operators and their layout are
// described there).
//
// Each 1D contraction is done by one thread per line: it keeps the line's
// inputs in registers and forms every output of the line as a dot product
// with a matrix row, read from shared memory as 16-byte broadcast vectors.
// That makes several multiply-adds per shared-memory load instead of one
// (the per-point form was bound by shared-memory instructions: LSU pipe 87%
// in FP32).  Stage work is shared between the three derivative directions:
//   divergence  X_D = Dg_i V, X_I = Ig_i V;  Y0 = Ig_j X_D, Y1 = Dg_j X_I,
//               Y2 = Ig_j X_I;  g_0 = Ig_k Y0, g_1 = Ig_k Y1, g_2 = Dg_k Y2
//   gradient    the transposes in reverse order, with the two terms that
//               meet Ig_i^T (from directions s and t) added before the last
//               contraction.
// EPB elements per CTA of 256 threads; tasks of a stage are strided over the
// CTA's threads.
#pragma once

namespace sem {
namespace pline {

constexpr int kThreads = 256;

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int W = 4;
};
template <>
struct Vec<double> {
  static constexpr int W = 2;
};

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// row[0..L) from shared memory, 16-byte aligned, as volatile vector loads (the
// compiler would otherwise hoist whole matrices into registers)
template <int L>
__device__ __forceinline__ void row_load(const float* p, float (&row)[L]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
#pragma unroll
  for (int c = 0; c < L; c += 4)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(row[c]), "=f"(row[c + 1]), "=f"(row[c + 2]), "=f"(row[c + 3])
                 : "r"(a + 4u * c));
}
template <int L>
__device__ __forceinline__ void row_load(const double* p, double (&row)[L]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
#pragma unroll
  for (int c = 0; c < L; c += 2)
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(row[c]), "=d"(row[c + 1]) : "r"(a + 8u * c));
}

// A hint to bring [p, p + bytes) into L2 (one bulk prefetch; nothing waits
// on it).  Skipped unless the range is 16-byte aligned at both ends.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  if (((uintptr_t)p & 15u) || (bytes & 15u) || bytes == 0 || bytes >= (1ull << 31)) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((uint32_t)bytes) : "memory");
}

template <typename T, int N>
struct Shape {
  static constexpr int n = N + 1, m = N - 1, n2 = n * n, n3 = n2 * n, m2 = m * m, m3 = m2 * m;
  static constexpr int W = Vec<T>::W;
  static constexpr int rn = round_up(n, W);  // padded row of an n -> m contraction matrix
  static constexpr int rm = round_up(m, W);  // padded row of an m -> n contraction matrix
  // Rows along i are padded by one (n + 1, m + 1 values): a thread per line
  // reads or writes its whole row, and the odd stride spreads a warp's rows
  // over the banks.  Per element: V or U [n^2][n + 1], two [n^2][m + 1],
  // three [n m^2], one [m^3].
  static constexpr int np1 = n + 1, mp1 = m + 1;
  static constexpr int elem = round_up(n2 * np1 + 2 * n2 * mp1 + 3 * n * m2 + m3, W);
  static constexpr int mats = 2 * m * rn + 2 * n * rm;  // Dg, Ig rows [m][rn]; Dg^T, Ig^T rows [n][rm]
  static constexpr int epb_raw = kThreads / n2 < 1 ? 1 : kThreads / n2;
  static constexpr int epb_cap = (int)((96 * 1024 / sizeof(T) - mats) / elem) < 1
                                     ? 1
                                     : (int)((96 * 1024 / sizeof(T) - mats) / elem);
  static constexpr int EPB = epb_raw < epb_cap ? (epb_raw < 16 ? epb_raw : 16) : epb_cap;
  static constexpr size_t smem = sizeof(T) * (size_t)(mats + EPB * elem);
};

// The four padded matrices: Dg, Ig rows [m][rn] and their transposes [n][rm].
template <typename T, int N>
__device__ __forceinline__ void load_mats(T* sm, const T* __restrict__ Ig, const T* __restrict__ DIg) {
  using S = Shape<T, N>;
  T* sDg = sm;
  T* sIg = sDg + S::m * S::rn;
  T* sDgT = sIg + S::m * S::rn;
  T* sIgT = sDgT + S::n * S::rm;
  for (int q = threadIdx.x; q < S::m * S::rn; q += blockDim.x) {
    const int r = q / S::rn, c = q % S::rn;
    sDg[q] = c < S::n ? DIg[r * S::n + c] : T(0);
    sIg[q] = c < S::n ? Ig[r * S::n + c] : T(0);
  }
  for (int q = threadIdx.x; q < S::n * S::rm; q += blockDim.x) {
    const int r = q / S::rm, c = q % S::rm;
    sDgT[q] = c < S::m ? DIg[c * S::n + r] : T(0);
    sIgT[q] = c < S::m ? Ig[c * S::n + r] : T(0);
  }
}

// out_q = sum_a sum_b F[b][a](q) (C_b v_a)(q), v_a = u_a / dB, u_a invB or u_a.
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_pdiv_line(const T* __restrict__ u, const T* __restrict__ dB,
                                                        const T* __restrict__ invB, const T* __restrict__ F,
                                                        const T* __restrict__ Ig, const T* __restrict__ DIg,
                                                        int64_t E, T* __restrict__ out, int64_t n_local) {
  using S = Shape<T, N>;
  constexpr int n = S::n, m = S::m, n2 = S::n2, n3 = S::n3, m2 = S::m2, m3 = S::m3, rn = S::rn, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  load_mats<T, N>(sm, Ig, DIg);
  const T* sDg = sm;
  const T* sIg = sDg + m * rn;
  T* el = sm + S::mats;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int ne = (int)min((int64_t)EPB, E - e0);
  // every F block and the later directions' velocity blocks are read only
  // after contractions: into L2 now
  if (threadIdx.x == 0) {
    prefetch_l2(F + e0 * 9 * m3, sizeof(T) * (size_t)ne * 9 * m3);
    prefetch_l2(u + n_local + e0 * n3, sizeof(T) * (size_t)ne * n3);
    prefetch_l2(u + 2 * n_local + e0 * n3, sizeof(T) * (size_t)ne * n3);
  }
  constexpr int np1 = S::np1, mp1 = S::mp1;
  auto V = [&](int le) { return el + le * S::elem; };
  auto XD = [&](int le) { return V(le) + n2 * np1; };
  auto XI = [&](int le) { return XD(le) + n2 * mp1; };
  auto Y0 = [&](int le) { return XI(le) + n2 * mp1; };
  auto Y1 = [&](int le) { return Y0(le) + n * m2; };
  auto Y2 = [&](int le) { return Y1(le) + n * m2; };
  auto O = [&](int le) { return Y2(le) + n * m2; };
  for (int a = 0; a < 3; ++a) {
    const T* ua = u + a * n_local + e0 * n3;
    for (int q = threadIdx.x; q < ne * n3; q += blockDim.x) {
      const int64_t g = e0 * n3 + q;
      const int r = q % n3;
      V(q / n3)[(r / n) * np1 + r % n] = dB ? ua[q] / dB[g] : (invB ? ua[q] * invB[g] : ua[q]);
    }
    __syncthreads();
    // stage 1, lines (k, j) along i: X_D = Dg V, X_I = Ig V
    for (int t = threadIdx.x; t < ne * n2; t += blockDim.x) {
      const int le = t / n2, kj = t % n2;
      const T* v = V(le) + kj * np1;
      T x[rn];
#pragma unroll
      for (int l = 0; l < rn; ++l) x[l] = l < n ? v[l] : T(0);
      T* xd = XD(le) + kj * mp1;
      T* xi = XI(le) + kj * mp1;
#pragma unroll
      for (int I = 0; I < m; ++I) {
        T rd[rn], ri[rn];
        row_load(sDg + I * rn, rd);
        row_load(sIg + I * rn, ri);
        T sd = T(0), si = T(0);
#pragma unroll
        for (int l = 0; l < rn; ++l) {
          sd += rd[l] * x[l];
          si += ri[l] * x[l];
        }
        xd[I] = sd;
        xi[I] = si;
      }
    }
    __syncthreads();
    // stage 2, lines (k, I) along j: Y0 = Ig X_D, Y1 = Dg X_I, Y2 = Ig X_I
    for (int t = threadIdx.x; t < ne * n * m; t += blockDim.x) {
      const int le = t / (n * m), kI = t % (n * m), k = kI / m, I = kI % m;
      const T* xd = XD(le) + k * n * mp1 + I;
      const T* xi = XI(le) + k * n * mp1 + I;
      T d[rn], c[rn];
#pragma unroll
      for (int j = 0; j < rn; ++j) {
        d[j] = j < n ? xd[j * mp1] : T(0);
        c[j] = j < n ? xi[j * mp1] : T(0);
      }
      T* y0 = Y0(le) + k * m2 + I;
      T* y1 = Y1(le) + k * m2 + I;
      T* y2 = Y2(le) + k * m2 + I;
#pragma unroll
      for (int J = 0; J < m; ++J) {
        T rd[rn], ri[rn];
        row_load(sDg + J * rn, rd);
        row_load(sIg + J * rn, ri);
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int j = 0; j < rn; ++j) {
          s0 += ri[j] * d[j];
          s1 += rd[j] * c[j];
          s2 += ri[j] * c[j];
        }
        y0[J * m] = s0;
        y1[J * m] = s1;
        y2[J * m] = s2;
      }
    }
    __syncthreads();
    // stage 3, lines (J, I) along k: g_b, combined with F[b][a] into O
    for (int t = threadIdx.x; t < ne * m2; t += blockDim.x) {
      const int le = t / m2, JI = t % m2;
      T c0[rn], c1[rn], c2[rn];
#pragma unroll
      for (int k = 0; k < rn; ++k) {
        c0[k] = k < n ? Y0(le)[k * m2 + JI] : T(0);
        c1[k] = k < n ? Y1(le)[k * m2 + JI] : T(0);
        c2[k] = k < n ? Y2(le)[k * m2 + JI] : T(0);
      }
      const T* Fe = F + (e0 + le) * 9 * m3 + JI;
      T* o = O(le) + JI;
#pragma unroll
      for (int K = 0; K < m; ++K) {
        T rd[rn], ri[rn];
        row_load(sDg + K * rn, rd);
        row_load(sIg + K * rn, ri);
        T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
        for (int k = 0; k < rn; ++k) {
          g0 += ri[k] * c0[k];
          g1 += ri[k] * c1[k];
          g2 += rd[k] * c2[k];
        }
        const int q = K * m2;
        const T v = Fe[(0 + a) * m3 + q] * g0 + Fe[(3 + a) * m3 + q] * g1 + Fe[(6 + a) * m3 + q] * g2;
        o[q] = a == 0 ? v : o[q] + v;
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < ne * m3; q += blockDim.x) out[e0 * m3 + q] = O(q / m3)[q % m3];
}

// u_a = sum_b C_b^T (F[b][a] p) for a = 0, 1, 2 (local, unassembled).
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_pgrad_line(const T* __restrict__ p, const T* __restrict__ F,
                                                         const T* __restrict__ Ig, const T* __restrict__ DIg,
                                                         int64_t E, T* __restrict__ u, int64_t n_local) {
  using S = Shape<T, N>;
  constexpr int n = S::n, m = S::m, n2 = S::n2, n3 = S::n3, m2 = S::m2, m3 = S::m3, rm = S::rm, rn = S::rn;
  constexpr int EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  load_mats<T, N>(sm, Ig, DIg);
  const T* sDgT = sm + 2 * m * rn;
  const T* sIgT = sDgT + n * rm;
  T* el = sm + S::mats;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int ne = (int)min((int64_t)EPB, E - e0);
  if (threadIdx.x == 0) prefetch_l2(F + e0 * 9 * m3, sizeof(T) * (size_t)ne * 9 * m3);
  // per element: U [n^2][n + 1], A0, A1 [n^2][m + 1], S0, S1, S2 [n m^2], P [m^3]
  constexpr int np1 = S::np1, mp1 = S::mp1;
  auto U = [&](int le) { return el + le * S::elem; };
  auto A0 = [&](int le) { return U(le) + n2 * np1; };
  auto A1 = [&](int le) { return A0(le) + n2 * mp1; };
  auto S0 = [&](int le) { return A1(le) + n2 * mp1; };
  auto S1 = [&](int le) { return S0(le) + n * m2; };
  auto S2 = [&](int le) { return S1(le) + n * m2; };
  auto P = [&](int le) { return S2(le) + n * m2; };
  for (int q = threadIdx.x; q < ne * m3; q += blockDim.x) P(q / m3)[q % m3] = p[e0 * m3 + q];
  __syncthreads();
  for (int a = 0; a < 3; ++a) {
    // stage 3', lines (J, I) along K -> k: S0 = Ig^T t0, S1 = Ig^T t1, S2 = Dg^T t2, t_b = F[b][a] p
    for (int t = threadIdx.x; t < ne * m2; t += blockDim.x) {
      const int le = t / m2, JI = t % m2;
      const T* Fe = F + (e0 + le) * 9 * m3 + JI;
      const T* pe = P(le) + JI;
      T t0[rm], t1[rm], t2[rm];
#pragma unroll
      for (int K = 0; K < rm; ++K) {
        const T pv = K < m ? pe[K * m2] : T(0);
        t0[K] = K < m ? Fe[(0 + a) * m3 + K * m2] * pv : T(0);
        t1[K] = K < m ? Fe[(3 + a) * m3 + K * m2] * pv : T(0);
        t2[K] = K < m ? Fe[(6 + a) * m3 + K * m2] * pv : T(0);
      }
      T* s0 = S0(le) + JI;
      T* s1 = S1(le) + JI;
      T* s2 = S2(le) + JI;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        T rd[rm], ri[rm];
        row_load(sDgT + k * rm, rd);
        row_load(sIgT + k * rm, ri);
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int K = 0; K < rm; ++K) {
          a0 += ri[K] * t0[K];
          a1 += ri[K] * t1[K];
          a2 += rd[K] * t2[K];
        }
        s0[k * m2] = a0;
        s1[k * m2] = a1;
        s2[k * m2] = a2;
      }
    }
    __syncthreads();
    // stage 2', lines (k, I) along J -> j: A0 = Ig^T S0, A1 = Dg^T S1 + Ig^T S2
    for (int t = threadIdx.x; t < ne * n * m; t += blockDim.x) {
      const int le = t / (n * m), kI = t % (n * m), k = kI / m, I = kI % m;
      const T* s0 = S0(le) + k * m2 + I;
      const T* s1 = S1(le) + k * m2 + I;
      const T* s2 = S2(le) + k * m2 + I;
      T c0[rm], c1[rm], c2[rm];
#pragma unroll
      for (int J = 0; J < rm; ++J) {
        c0[J] = J < m ? s0[J * m] : T(0);
        c1[J] = J < m ? s1[J * m] : T(0);
        c2[J] = J < m ? s2[J * m] : T(0);
      }
      T* a0 = A0(le) + k * n * mp1 + I;
      T* a1 = A1(le) + k * n * mp1 + I;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        T rd[rm], ri[rm];
        row_load(sDgT + j * rm, rd);
        row_load(sIgT + j * rm, ri);
        T v0 = T(0), v1 = T(0);
#pragma unroll
        for (int J = 0; J < rm; ++J) {
          v0 += ri[J] * c0[J];
          v1 += rd[J] * c1[J] + ri[J] * c2[J];
        }
        a0[j * mp1] = v0;
        a1[j * mp1] = v1;
      }
    }
    __syncthreads();
    // stage 1', lines (k, j) along I -> i: U = Dg^T A0 + Ig^T A1
    for (int t = threadIdx.x; t < ne * n2; t += blockDim.x) {
      const int le = t / n2, kj = t % n2;
      const T* x0 = A0(le) + kj * mp1;
      const T* x1 = A1(le) + kj * mp1;
      T c0[rm], c1[rm];
#pragma unroll
      for (int I = 0; I < rm; ++I) {
        c0[I] = I < m ? x0[I] : T(0);
        c1[I] = I < m ? x1[I] : T(0);
      }
      T* uu = U(le) + kj * np1;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        T rd[rm], ri[rm];
        row_load(sDgT + i * rm, rd);
        row_load(sIgT + i * rm, ri);
        T v = T(0);
#pragma unroll
        for (int I = 0; I < rm; ++I) v += rd[I] * c0[I] + ri[I] * c1[I];
        uu[i] = v;
      }
    }
    __syncthreads();
    T* ua = u + a * n_local + e0 * n3;
    for (int q = threadIdx.x; q < ne * n3; q += blockDim.x) {
      const int r = q % n3;
      ua[q] = U(q / n3)[(r / n) * np1 + r % n];
    }
    // the next direction rewrites S (read in stage 2', done) and U (read just now)
    __syncthreads();
  }
}

}  // namespace pline
}  // namespace sem
