// Device kernels of the overlapping Schwarz preconditioner (Sec. 2, Eq. 6):
//
//   M^{-1} r = mask QQ^T (W A~_e^{-1} (W r_e) for every element e)  +  R_0^T A_0^{-1} R_0 r
//
// Local solves: each subdomain is one element with all its GLL nodes (the
// overlap is the nodes it shares), its problem replaced by the separable
// fast-diagonalisation form
//   A~_e^{-1} = (S_t (x) S_s (x) S_r) (h1 (lam_r + lam_s + lam_t) + h2)^{-1} (S_t (x) S_s (x) S_r)^T
// with per-element 1D eigenpairs (S, lam) built on the host; W = mult^{-1/2}
// on both sides (the symmetric weighting).  The coarse space is the trilinear
// functions of the element vertices: R_0 restricts (each global node once),
// A_0 = R_0 A R_0^T is assembled from 8 x 8 element matrices, and R_0^T
// interpolates the vertex values back to the GLL points.
//
// Thread mapping of the local solve: as the local operator, a thread owns one
// (i, j) column of an element and keeps it in registers, so the t-direction
// contractions never touch shared memory; r and s go through two padded n^3
// arrays per element.  Per point 6n multiply-adds (n per contraction).
#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "sem_internal.h"
#include "schwarz.h"

namespace sem {

namespace {

// Shared-memory layout of one element's n^3 values for the line-based local
// solve.  Each contraction has a thread per line of its direction: r-lines
// (fixed j, k), s-lines (fixed i, k) and t-lines (fixed i, j), so the three
// access patterns of a warp are (j, k), (i, k) and (i, j) varying with the
// third index fixed.  n = 8, FP32: rows of 8, planes padded to 72, and i
// XOR-swizzled by f(j, k) = (2k + j / 4) mod 8, which puts the 32 lanes of all
// three patterns on 32 distinct banks.  Other cases: rows padded to n + 1 and
// planes to n (n + 1) + 1.
template <int n, typename T>
struct FdmLay {
  static constexpr bool swz = (n == 8) && sizeof(T) == 4;
  static constexpr int RP = swz ? 8 : n + 1;
  static constexpr int PL = swz ? 72 : n * (n + 1) + 1;
  static constexpr int size = n * PL;
  __device__ static __forceinline__ int idx(int i, int j, int k) {
    if constexpr (swz) return k * PL + j * RP + (i ^ ((2 * k + (j >> 2)) & 7));
    return k * PL + j * RP + i;
  }
};

// Rows of the 1D matrices are read with volatile vector loads from shared
// memory, at the point of use: the compiler then neither hoists the whole
// n x n matrix into registers (110 registers at N = 7 with plain loads, two
// CTAs per SM) nor merges the loads of the forward and back contractions.
__device__ __forceinline__ float4 lds4(const float* p) {
  float4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ double2 lds2(const double* p) {
  double2 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
  return v;
}

// row[0..n) = S[r * n .. r * n + n) (16-byte aligned rows when n is a multiple
// of the vector width; scalar loads otherwise)
template <int n, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ S, int r, T (&row)[n]) {
  if constexpr (sizeof(T) == 4 && n % 4 == 0) {
#pragma unroll
    for (int c = 0; c < n; c += 4) {
      const float4 v = lds4(reinterpret_cast<const float*>(S) + r * n + c);
      row[c] = v.x, row[c + 1] = v.y, row[c + 2] = v.z, row[c + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 8 && n % 2 == 0) {
#pragma unroll
    for (int c = 0; c < n; c += 2) {
      const double2 v = lds2(reinterpret_cast<const double*>(S) + r * n + c);
      row[c] = v.x, row[c + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < n; ++c) row[c] = S[r * n + c];
  }
}

// out[c] = sum_l S[l][c] x[l] (trans = false) or sum_l S[c][l] x[l] (trans =
// true) for the n x n matrix S in shared memory, rows read as broadcasts.
template <int n, typename T, bool TRANS>
__device__ __forceinline__ void line_contract(const T* __restrict__ S, const T (&x)[n], T (&out)[n]) {
#pragma unroll
  for (int c = 0; c < n; ++c) out[c] = T(0);
  T row[n];
  if constexpr (!TRANS) {
#pragma unroll
    for (int l = 0; l < n; ++l) {
      load_row<n, T>(S, l, row);
#pragma unroll
      for (int c = 0; c < n; ++c) out[c] += row[c] * x[l];
    }
  } else {
#pragma unroll
    for (int c = 0; c < n; ++c) {
      load_row<n, T>(S, c, row);
#pragma unroll
      for (int l = 0; l < n; ++l) out[c] += row[l] * x[l];
    }
  }
}

// (With the 1D matrices hoisted into registers, 110 registers at N = 7 in
// FP32; forcing three CTAs per SM then spilled and measured slower, 1.43 ms
// instead of 1.32 ms for one FP32 application at E = 262,144.)
template <int N, typename T, int EPB>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1)) k_fdm(const FdmParams<T> P) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  using L = FdmLay<n, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sS = reinterpret_cast<T*>(smem_raw);  // [EPB][3][n][n]: S_r, S_s, S_t (row l, column = eigenvector)
  T* sL = sS + EPB * 3 * n2;               // [EPB][3][n]
  T* sX = sL + EPB * 3 * n;                // [EPB][L::size]
  T* sR = sX + EPB * L::size;              // [EPB][8][n^2]: coarse restriction, per column (P.rc only)
  __shared__ int sdone;
  const int tid = threadIdx.x;
  if (P.st) {
    if (tid == 0) sdone = P.st->done;
    __syncthreads();
    if (sdone) return;
  }
  const int le = tid / n2, q = tid - le * n2;
  const int a = q % n, b = q / n;  // this thread's line: (a, b) = the two fixed indices
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool act = e < P.E;
  T* Se = sS + le * 3 * n2;
  T* Le = sL + le * 3 * n;
  T* X = sX + le * L::size;
  if (act) {
    for (int t = q; t < 3 * n2; t += n2) {
      const int d = t / n2;
      Se[t] = P.S[(int64_t)P.sidx[3 * e + d] * n2 + (t - d * n2)];
    }
    for (int t = q; t < 3 * n; t += n2) {
      const int d = t / n;
      Le[t] = P.lam[(int64_t)P.sidx[3 * e + d] * n + (t - d * n)];
    }
  }
  // W r, coalesced: thread q holds point (i, j) = (a, b) of every k-plane
  const int64_t base = e * n3 + q;
  if (act) {
    T t0 = T(0), t1 = T(0);  // coarse restriction of this column: sum_k f_b(xi_k) r / mult
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const T wk = P.wtab[P.wm[base + k * n2] & 0x7f];
      const T wr = wk * P.r[base + k * n2];
      X[L::idx(a, b, k)] = wr;
      if (P.rc) {
        const T rm = wk * wr;  // r / mult
        t0 += P.ftab[k] * rm;
        t1 += P.ftab[n + k] * rm;
      }
    }
    if (P.rc) {
      T* R = sR + le * 8 * n2;
      const T fa[2] = {P.ftab[a], P.ftab[n + a]}, fb[2] = {P.ftab[b], P.ftab[n + b]};
#pragma unroll
      for (int v = 0; v < 8; ++v) R[v * n2 + q] = fa[v & 1] * fb[(v >> 1) & 1] * ((v >> 2) & 1 ? t1 : t0);
    }
  }
  __syncthreads();
  if (P.rc && act) {  // one thread per element vertex: the element's columns in order
    for (int v = q; v < 8; v += n2) {
      const T* R = sR + le * 8 * n2 + v * n2;
      T sum = T(0);
      for (int c = 0; c < n2; ++c) sum += R[c];
      P.rc[8 * e + v] = (double)sum;
    }
  }
  T x[n], y[n];
  // forward r: line (j, k) = (a, b)
  if (act) {
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = X[L::idx(l, a, b)];
    line_contract<n, T, false>(Se, x, y);
#pragma unroll
    for (int l = 0; l < n; ++l) X[L::idx(l, a, b)] = y[l];
  }
  __syncthreads();
  // forward s: line (i, k) = (a, b)
  if (act) {
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = X[L::idx(a, l, b)];
    line_contract<n, T, false>(Se + n2, x, y);
#pragma unroll
    for (int l = 0; l < n; ++l) X[L::idx(a, l, b)] = y[l];
  }
  __syncthreads();
  // t: line (i, j) = (a, b): forward, divide by h1 (lam_r + lam_s + lam_t) + h2, back
  if (act) {
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = X[L::idx(a, b, l)];
    line_contract<n, T, false>(Se + 2 * n2, x, y);
    const T lab = Le[a] + Le[n + b];
#pragma unroll
    for (int l = 0; l < n; ++l) y[l] = y[l] / (P.h1 * (lab + Le[2 * n + l]) + P.h2);
    line_contract<n, T, true>(Se + 2 * n2, y, x);
#pragma unroll
    for (int l = 0; l < n; ++l) X[L::idx(a, b, l)] = x[l];
  }
  __syncthreads();
  // back s: line (i, k) = (a, b)
  if (act) {
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = X[L::idx(a, l, b)];
    line_contract<n, T, true>(Se + n2, x, y);
#pragma unroll
    for (int l = 0; l < n; ++l) X[L::idx(a, l, b)] = y[l];
  }
  __syncthreads();
  // back r: line (j, k) = (a, b)
  if (act) {
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = X[L::idx(l, a, b)];
    line_contract<n, T, true>(Se, x, y);
#pragma unroll
    for (int l = 0; l < n; ++l) X[L::idx(l, a, b)] = y[l];
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int k = 0; k < n; ++k) P.z[base + k * n2] = P.wtab[P.wm[base + k * n2] & 0x7f] * X[L::idx(a, b, k)];
  }
}

template <int N, typename T, int EPB>
size_t fdm_smem() {
  constexpr int n = N + 1;
  return sizeof(T) * ((size_t)EPB * (3 * n * n + 3 * n) + (size_t)EPB * FdmLay<n, T>::size + 8ull * EPB * n * n);
}

template <int N, typename T>
cudaError_t launch_fdm_n(const FdmParams<T>& p, cudaStream_t s) {
  constexpr int n = N + 1;
  constexpr int EPB = (256 / (n * n)) < 1 ? 1 : 256 / (n * n);
  const size_t smem = fdm_smem<N, T, EPB>();
  static DeviceOnce once;
  cudaError_t err = once.get([&](int, int*) {
    return cudaFuncSetAttribute(k_fdm<N, T, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (err != cudaSuccess) return err;
  if (p.E == 0) return cudaSuccess;
  const int64_t grid = (p.E + EPB - 1) / EPB;
  k_fdm<N, T, EPB><<<(unsigned)grid, EPB * n * n, smem, s>>>(p);
  return cudaGetLastError();
}

// ---- coarse space -------------------------------------------------------------
//
// Vertex v of an element is (bi, bj, bk) = (v & 1, (v >> 1) & 1, (v >> 2) & 1);
// its function at GLL point (i, j, k) is f_bi(xi_i) f_bj(xi_j) f_bk(xi_k) with
// f_0 = (1 - xi) / 2 and f_1 = (1 + xi) / 2.

// rc[8 e + v] = rscale * (sum over the element's points of phi_v r / mult).
// ftab [2][n] = f_0, f_1 at the GLL nodes in T.  A thread owns one (i, j)
// column: t_b = sum_k f_b(xi_k) r / mult (2 multiply-adds per point in T),
// then c_v = f_bi(xi_i) f_bj(xi_j) t_bk, summed over the element's columns in
// a fixed order (shared memory, one warp per element-vertex pair).
template <typename T, int EPB>
__global__ void k_coarse_restrict(const T* __restrict__ r, const uint8_t* __restrict__ wm, const T* __restrict__ ftab,
                                  int n, int64_t E, double rscale, double* __restrict__ rc, const PcgState* st) {
  extern __shared__ double scol[];  // [EPB][8][n^2]
  __shared__ T sinv[128];
  __shared__ int sdone;
  const int n2 = n * n, n3 = n2 * n;
  for (int m = threadIdx.x; m < 128; m += blockDim.x) sinv[m] = m ? T(1) / T(m) : T(0);
  if (threadIdx.x == 0) sdone = st ? st->done : 0;
  __syncthreads();
  if (sdone) return;
  const int le = threadIdx.x / n2, ij = threadIdx.x - le * n2, i = ij % n, j = ij / n;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  double* col = scol + (size_t)le * 8 * n2;
  if (le < EPB) {
    T t0 = T(0), t1 = T(0);
    if (e < E) {
      for (int k = 0; k < n; ++k) {
        const int64_t q = e * n3 + k * n2 + ij;
        const T val = r[q] * sinv[wm[q] & 0x7f];
        t0 += ftab[k] * val;
        t1 += ftab[n + k] * val;
      }
    }
#pragma unroll
    for (int v = 0; v < 8; ++v)
      col[v * n2 + ij] = (double)(ftab[(v & 1) * n + i] * ftab[((v >> 1) & 1) * n + j] * ((v >> 2) & 1 ? t1 : t0));
  }
  __syncthreads();
  // one warp per (element, vertex): fixed lane ranges, fixed shuffle tree
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int ev = warp; ev < EPB * 8; ev += nw) {
    const int le2 = ev >> 3, v = ev & 7;
    const int64_t e2 = (int64_t)blockIdx.x * EPB + le2;
    const double* c = scol + (size_t)le2 * 8 * n2 + v * n2;
    double s = 0.0;
    for (int q = lane; q < n2; q += 32) s += c[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0 && e2 < E) rc[8 * e2 + v] = s * rscale;
  }
}

// g[c] = sum of rc over the (element, vertex) slots of coarse unknown c, in
// ascending slot order (CSR lists from the host).
__global__ void k_coarse_gather(const double* __restrict__ rc, const int32_t* __restrict__ ptr,
                                const int64_t* __restrict__ slots, int nc, double* __restrict__ g,
                                const PcgState* st) {
  if (st && st->done) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = ptr[c]; q < ptr[c + 1]; ++q) s += rc[slots[q]];
    g[c] = s;
  }
}

// y = A y_in for the dense symmetric matrix A (row-major, nc x nc): one warp
// per row, fixed lane ranges and a fixed shuffle tree (deterministic).
__global__ void k_dense_symv(const double* __restrict__ A, const double* __restrict__ x, int nc,
                             double* __restrict__ y, const PcgState* st) {
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nc; row += warps) {
    const double* a = A + (int64_t)row * nc;
    double s = 0.0;
    for (int c = lane; c < nc; c += 32) s += a[c] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
  }
}

// z += zscale * mask R_0^T y: the trilinear interpolant of the element's
// vertex values (0 at Dirichlet vertices, cidx < 0) at every GLL point.  A
// thread owns one (i, j) column: a_bk = sum_{bi,bj} f_bi(xi_i) f_bj(xi_j)
// y_v, then z += f_0(xi_k) a_0 + f_1(xi_k) a_1 (2 multiply-adds per point in T).
template <typename T, int EPB>
__global__ void k_coarse_prolong(T* __restrict__ z, const uint8_t* __restrict__ wm, const T* __restrict__ ftab,
                                 const int32_t* __restrict__ cidx, const double* __restrict__ y, int n, int64_t E,
                                 double zscale, const PcgState* st) {
  __shared__ T cv[EPB][8];
  __shared__ int sdone;
  const int n2 = n * n, n3 = n2 * n;
  if (threadIdx.x == 0) sdone = st ? st->done : 0;
  if (threadIdx.x < 8 * EPB) {
    const int64_t e = (int64_t)blockIdx.x * EPB + threadIdx.x / 8;
    const int c = e < E ? cidx[8 * e + (threadIdx.x & 7)] : -1;
    cv[threadIdx.x / 8][threadIdx.x & 7] = c >= 0 ? (T)(y[c] * zscale) : T(0);
  }
  __syncthreads();
  if (sdone) return;
  const int le = threadIdx.x / n2, ij = threadIdx.x - le * n2, i = ij % n, j = ij / n;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  if (le >= EPB || e >= E) return;
  const T* c = cv[le];
  const T fi0 = ftab[i], fi1 = ftab[n + i], fj0 = ftab[j], fj1 = ftab[n + j];
  const T a0 = fj0 * (fi0 * c[0] + fi1 * c[1]) + fj1 * (fi0 * c[2] + fi1 * c[3]);
  const T a1 = fj0 * (fi0 * c[4] + fi1 * c[5]) + fj1 * (fi0 * c[6] + fi1 * c[7]);
  for (int k = 0; k < n; ++k) {
    const int64_t q = e * n3 + k * n2 + ij;
    if (wm[q] & 0x80) continue;  // Dirichlet: the masked field is 0 there
    z[q] = z[q] + (ftab[k] * a0 + ftab[n + k] * a1);
  }
}

// z += mask R_0^T y, then <r, z>_W: a grid-stride loop over element groups
// (fixed per block), compensated FP32 or FP64 sums per thread, fixed-order
// block sums and a last-block sum of the block partials (deterministic).
struct RhoAcc64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};
struct RhoAccF32 {  // Knuth's TwoSum on the FP32 pipe
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

// RHO = false: only z += mask R_0^T y (st nullable, r unused).
template <typename T, int n, int EPB, bool RHO>
__global__ void __launch_bounds__(((EPB * n * n + 31) / 32) * 32)
    k_prolong_rho(T* __restrict__ z, const T* __restrict__ r, const uint8_t* __restrict__ wm,
                  const T* __restrict__ ftab, const int32_t* __restrict__ cidx, const double* __restrict__ y,
                  int64_t E, PcgState* st, double* __restrict__ partial) {
  using Acc = typename std::conditional<std::is_same<T, float>::value, RhoAccF32, RhoAcc64>::type;
  constexpr int n2 = n * n, n3 = n2 * n;
  __shared__ T cv[EPB][8];
  __shared__ T sinv[128];
  __shared__ double sred[32];
  __shared__ int sdone;
  if (threadIdx.x == 0) sdone = st ? st->done : 0;
  if (RHO)
    for (int m = threadIdx.x; m < 128; m += blockDim.x) sinv[m] = m ? T(1) / T(m) : T(0);
  __syncthreads();
  if (sdone) return;
  const int le = threadIdx.x / n2, ij = threadIdx.x - le * n2, i = ij % n, j = ij / n;
  const int64_t groups = (E + EPB - 1) / EPB;
  Acc acc;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    for (int t = threadIdx.x; t < 8 * EPB; t += blockDim.x) {
      const int64_t e = g * EPB + t / 8;
      const int c = e < E ? cidx[8 * e + (t & 7)] : -1;
      cv[t / 8][t & 7] = c >= 0 ? (T)y[c] : T(0);
    }
    const int64_t e = g * EPB + le;
    const bool act = le < EPB && e < E;
    // this column's n values of z, r and the point flags, all loads in flight together
    T zv[n], rv[n];
    uint8_t mv[n];
    if (act) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int64_t q = e * n3 + k * n2 + ij;
        zv[k] = z[q];
        rv[k] = RHO ? r[q] : T(0);
        mv[k] = wm[q];
      }
    }
    __syncthreads();  // cv filled
    if (act) {
      const T* c = cv[le];
      const T fi0 = ftab[i], fi1 = ftab[n + i], fj0 = ftab[j], fj1 = ftab[n + j];
      const T a0 = fj0 * (fi0 * c[0] + fi1 * c[1]) + fj1 * (fi0 * c[2] + fi1 * c[3]);
      const T a1 = fj0 * (fi0 * c[4] + fi1 * c[5]) + fj1 * (fi0 * c[6] + fi1 * c[7]);
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int64_t q = e * n3 + k * n2 + ij;
        T zq = zv[k];
        if (!(mv[k] & 0x80)) {  // Dirichlet points keep z (0 there)
          zq = zq + (ftab[k] * a0 + ftab[n + k] * a1);
          z[q] = zq;
        }
        if (RHO) acc.add(rv[k] * zq * sinv[mv[k] & 0x7f]);
      }
    }
    __syncthreads();  // cv is rewritten for the next group
  }
  if (!RHO) return;
  const double a = block_sum(acc.get(), sred);
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

// u = mask phi_b on every element (the b-th vertex function, set-up only).
__global__ void k_fill_phi(double* __restrict__ u, const uint8_t* __restrict__ wm, const double* __restrict__ xi,
                           int n, int64_t P, int b) {
  const int n2 = n * n, n3 = n2 * n;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(p % n3);
    const int i = q % n, j = (q / n) % n, k = q / n2;
    const double fi = (b & 1) ? 0.5 * (1.0 + xi[i]) : 0.5 * (1.0 - xi[i]);
    const double fj = ((b >> 1) & 1) ? 0.5 * (1.0 + xi[j]) : 0.5 * (1.0 - xi[j]);
    const double fk = ((b >> 2) & 1) ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
    u[p] = (wm[p] & 0x80) ? 0.0 : fk * fj * fi;
  }
}

// Ae[e][a][b] = sum over the element's points of (mask phi_a) w, w = A_L (mask phi_b).
__global__ void k_elem_coarse(const double* __restrict__ w, const uint8_t* __restrict__ wm,
                              const double* __restrict__ xi, int n, int b, double* __restrict__ Ae) {
  __shared__ double sred[32];
  const int64_t e = blockIdx.x;
  const int n2 = n * n, n3 = n2 * n;
  double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int q = threadIdx.x; q < n3; q += blockDim.x) {
    if (wm[e * n3 + q] & 0x80) continue;
    const int i = q % n, j = (q / n) % n, k = q / n2;
    const double fi[2] = {0.5 * (1.0 - xi[i]), 0.5 * (1.0 + xi[i])};
    const double fj[2] = {0.5 * (1.0 - xi[j]), 0.5 * (1.0 + xi[j])};
    const double fk[2] = {0.5 * (1.0 - xi[k]), 0.5 * (1.0 + xi[k])};
    const double val = w[e * n3 + q];
#pragma unroll
    for (int a = 0; a < 8; ++a) c[a] += fk[(a >> 2) & 1] * fj[(a >> 1) & 1] * fi[a & 1] * val;
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const double s = block_sum(c[a], sred);
    if (threadIdx.x == 0) Ae[64 * e + 8 * a + b] = s;
  }
}

// One step k of Gauss-Jordan inversion of a symmetric positive definite
// matrix in place (no pivoting: the pivots of an SPD matrix stay positive).
// Step a (one CTA): f[i] = M[i][k] (the old column), then row k scaled by
// p = 1 / M[k][k] with M[k][k] = p.  Step b: every other row i,
// M[i][j] -= f[i] M[k][j] (j != k) and M[i][k] = -f[i] p.
__global__ void k_gj_pivot(double* __restrict__ M, int nc, int k, double* __restrict__ f, int* bad) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) f[i] = M[(int64_t)i * nc + k];
  __syncthreads();
  const double piv = f[k];
  if (!(piv > 0.0)) {
    if (threadIdx.x == 0) *bad = 1;
    return;
  }
  const double p = 1.0 / piv;
  for (int j = threadIdx.x; j < nc; j += blockDim.x) M[(int64_t)k * nc + j] = (j == k) ? p : M[(int64_t)k * nc + j] * p;
}
__global__ void k_gj_update(double* __restrict__ M, int nc, int k, const double* __restrict__ f) {
  const int64_t total = (int64_t)nc * nc;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / nc), j = (int)(q - (int64_t)i * nc);
    if (i == k) continue;
    const double mk = M[(int64_t)k * nc + j];
    M[q] = (j == k) ? -f[i] * mk : M[q] - f[i] * mk;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_fdm(int N, const FdmParams<T>& p, cudaStream_t s) {
  switch (N) {
    case 1: return launch_fdm_n<1, T>(p, s);
    case 2: return launch_fdm_n<2, T>(p, s);
    case 3: return launch_fdm_n<3, T>(p, s);
    case 4: return launch_fdm_n<4, T>(p, s);
    case 5: return launch_fdm_n<5, T>(p, s);
    case 6: return launch_fdm_n<6, T>(p, s);
    case 7: return launch_fdm_n<7, T>(p, s);
    case 8: return launch_fdm_n<8, T>(p, s);
    case 9: return launch_fdm_n<9, T>(p, s);
    case 10: return launch_fdm_n<10, T>(p, s);
    case 11: return launch_fdm_n<11, T>(p, s);
    default: return cudaErrorNotSupported;
  }
}
template cudaError_t launch_fdm<double>(int, const FdmParams<double>&, cudaStream_t);
template cudaError_t launch_fdm<float>(int, const FdmParams<float>&, cudaStream_t);

template <typename T>
cudaError_t launch_coarse_restrict(const T* r, const uint8_t* wm, const T* ftab, int n, int64_t E, double rscale,
                                   double* rc, const PcgState* st, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  constexpr int EPB = 4;  // n <= 8: 4 elements of n^2 <= 64 columns; larger n: one element per CTA
  if (n <= 8) {
    const size_t smem = sizeof(double) * 8 * EPB * n * n;
    const unsigned threads = ((EPB * n * n + 31) / 32) * 32;
    k_coarse_restrict<T, EPB><<<(unsigned)((E + EPB - 1) / EPB), threads, smem, s>>>(r, wm, ftab, n, E, rscale, rc, st);
  } else {
    const size_t smem = sizeof(double) * 8 * n * n;
    const unsigned threads = ((n * n + 31) / 32) * 32;
    k_coarse_restrict<T, 1><<<(unsigned)E, threads, smem, s>>>(r, wm, ftab, n, E, rscale, rc, st);
  }
  return cudaGetLastError();
}
template cudaError_t launch_coarse_restrict<double>(const double*, const uint8_t*, const double*, int, int64_t, double,
                                                    double*, const PcgState*, cudaStream_t);
template cudaError_t launch_coarse_restrict<float>(const float*, const uint8_t*, const float*, int, int64_t, double,
                                                   double*, const PcgState*, cudaStream_t);

cudaError_t launch_coarse_gather(const double* rc, const int32_t* ptr, const int64_t* slots, int nc, double* g,
                                 const PcgState* st, cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  const int blocks = std::min(1024, (nc + 255) / 256);
  k_coarse_gather<<<blocks, 256, 0, s>>>(rc, ptr, slots, nc, g, st);
  return cudaGetLastError();
}

cudaError_t launch_dense_symv(const double* A, const double* x, int nc, double* y, const PcgState* st, cudaStream_t s) {
  if (nc == 0) return cudaSuccess;
  const int blocks = std::min(152 * 8, (nc + 7) / 8);
  k_dense_symv<<<blocks, 256, 0, s>>>(A, x, nc, y, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_prolong(T* z, const uint8_t* wm, const T* ftab, const int32_t* cidx, const double* y, int n,
                                  int64_t E, double zscale, const PcgState* st, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  constexpr int EPB = 4;
  if (n <= 8) {
    const unsigned threads = ((EPB * n * n + 31) / 32) * 32;
    k_coarse_prolong<T, EPB><<<(unsigned)((E + EPB - 1) / EPB), threads, 0, s>>>(z, wm, ftab, cidx, y, n, E, zscale, st);
  } else {
    const unsigned threads = ((n * n + 31) / 32) * 32;
    k_coarse_prolong<T, 1><<<(unsigned)E, threads, 0, s>>>(z, wm, ftab, cidx, y, n, E, zscale, st);
  }
  return cudaGetLastError();
}
template cudaError_t launch_coarse_prolong<double>(double*, const uint8_t*, const double*, const int32_t*,
                                                   const double*, int, int64_t, double, const PcgState*, cudaStream_t);
template cudaError_t launch_coarse_prolong<float>(float*, const uint8_t*, const float*, const int32_t*, const double*,
                                                  int, int64_t, double, const PcgState*, cudaStream_t);

template <typename T, int n>
cudaError_t launch_prolong_rho_n(T* z, const T* r, const uint8_t* wm, const T* ftab, const int32_t* cidx,
                                 const double* y, int64_t E, PcgState* st, double* partial, cudaStream_t s) {
  constexpr int EPB = (256 / (n * n)) < 1 ? 1 : 256 / (n * n);
  const int grid = (int)std::min<int64_t>(152 * 4, std::max<int64_t>(1, (E + EPB - 1) / EPB));  // <= the partials
  if (partial)
    k_prolong_rho<T, n, EPB, true><<<grid, ((EPB * n * n + 31) / 32) * 32, 0, s>>>(z, r, wm, ftab, cidx, y, E, st,
                                                                                  partial);
  else
    k_prolong_rho<T, n, EPB, false><<<grid, ((EPB * n * n + 31) / 32) * 32, 0, s>>>(z, r, wm, ftab, cidx, y, E, st,
                                                                                   partial);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_rho(T* z, const T* r, const uint8_t* wm, const T* ftab, const int32_t* cidx,
                               const double* y, int n, int64_t E, PcgState* st, double* partial, cudaStream_t s) {
  switch (n) {
    case 2: return launch_prolong_rho_n<T, 2>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 3: return launch_prolong_rho_n<T, 3>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 4: return launch_prolong_rho_n<T, 4>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 5: return launch_prolong_rho_n<T, 5>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 6: return launch_prolong_rho_n<T, 6>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 7: return launch_prolong_rho_n<T, 7>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 8: return launch_prolong_rho_n<T, 8>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 9: return launch_prolong_rho_n<T, 9>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 10: return launch_prolong_rho_n<T, 10>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 11: return launch_prolong_rho_n<T, 11>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    case 12: return launch_prolong_rho_n<T, 12>(z, r, wm, ftab, cidx, y, E, st, partial, s);
    default: return cudaErrorNotSupported;
  }
}
template cudaError_t launch_prolong_rho<double>(double*, const double*, const uint8_t*, const double*, const int32_t*,
                                                const double*, int, int64_t, PcgState*, double*, cudaStream_t);
template cudaError_t launch_prolong_rho<float>(float*, const float*, const uint8_t*, const float*, const int32_t*,
                                               const double*, int, int64_t, PcgState*, double*, cudaStream_t);

cudaError_t launch_fill_phi(double* u, const uint8_t* wm, const double* xi, int n, int64_t P, int b, cudaStream_t s) {
  k_fill_phi<<<152 * 8, 256, 0, s>>>(u, wm, xi, n, P, b);
  return cudaGetLastError();
}

cudaError_t launch_elem_coarse(const double* w, const uint8_t* wm, const double* xi, int n, int64_t E, int b,
                               double* Ae, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_elem_coarse<<<(unsigned)E, 128, 0, s>>>(w, wm, xi, n, b, Ae);
  return cudaGetLastError();
}

cudaError_t launch_gj_inverse(double* M, int nc, double* f, int* bad, cudaStream_t s) {
  const int64_t total = (int64_t)nc * nc;
  const int blocks = (int)std::min<int64_t>(152 * 8, (total + 255) / 256);
  for (int k = 0; k < nc; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(M, nc, k, f, bad);
    k_gj_update<<<blocks, 256, 0, s>>>(M, nc, k, f);
  }
  return cudaGetLastError();
}

// ---- coarse problem of many unknowns: a symmetric two-level cycle -----------
//
// A_0 (CSR) is solved approximately by one symmetric V-cycle: Chebyshev
// smoothing in D^{-1} A_0 (degree deg, zero start), the aggregate correction
// P A_00^{-1} P^T of the residual (P: piecewise constant on aggregates, A_00 =
// P^T A_0 P inverted densely), and the same Chebyshev smoothing again.  Every
// step is linear and the cycle symmetric, so the preconditioner stays a fixed
// SPD operator and CG keeps its recurrences.

namespace {

// A_0 is stored in ELL form, slot-major: row i's k-th entry at k * nc + i
// (val, col; unused slots hold 0 and column i), so one thread per row reads
// each slot coalesced across the rows of a warp, in a fixed order.

// d = c0 dinv r; x = d (acc = 0) or x += d (acc = 1); rcopy = r (nullable)
__global__ void k_cheb_first(const double* __restrict__ r, const double* __restrict__ dinv, double c0,
                             double* __restrict__ d, double* __restrict__ x, double* __restrict__ rcopy, int nc,
                             int acc, const PcgState* st) {
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const double ri = r[i];
    const double v = c0 * dinv[i] * ri;
    d[i] = v;
    x[i] = acc ? x[i] + v : v;
    if (rcopy) rcopy[i] = ri;
  }
}

// r -= A d_prev; d_new = a d_prev + b dinv r; x += d_new (one thread per row)
__global__ void k_cheb_step(const int32_t* __restrict__ col, const double* __restrict__ val, int width,
                            const double* __restrict__ dinv, const double* __restrict__ dprev,
                            double* __restrict__ dnew, double* __restrict__ r, double* __restrict__ x, double a,
                            double b, int nc, const PcgState* st) {
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < width; ++k) s += val[(int64_t)k * nc + i] * dprev[col[(int64_t)k * nc + i]];
    const double ri = r[i] - s;
    r[i] = ri;
    const double dn = a * dprev[i] + b * dinv[i] * ri;
    dnew[i] = dn;
    x[i] += dn;
  }
}

// r = g - A x
__global__ void k_ell_resid(const int32_t* __restrict__ col, const double* __restrict__ val, int width,
                            const double* __restrict__ g, const double* __restrict__ x, double* __restrict__ r, int nc,
                            const PcgState* st) {
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < width; ++k) s += val[(int64_t)k * nc + i] * x[col[(int64_t)k * nc + i]];
    r[i] = g[i] - s;
  }
}

// ga[a] = sum of r over the members of aggregate a (ascending)
__global__ void k_agg_restrict(const int32_t* __restrict__ aptr, const int32_t* __restrict__ amem,
                               const double* __restrict__ r, double* __restrict__ ga, int na, const PcgState* st) {
  if (st && st->done) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = aptr[a]; q < aptr[a + 1]; ++q) s += r[amem[q]];
    ga[a] = s;
  }
}

// x += ya[agg]
__global__ void k_agg_prolong(const int32_t* __restrict__ agg, const double* __restrict__ ya, double* __restrict__ x,
                              int nc, const PcgState* st) {
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) x[i] += ya[agg[i]];
}

int vgrid(int nc) { return std::max(1, std::min(152 * 16, (nc + 255) / 256)); }

}  // namespace

cudaError_t launch_vcycle(const CoarseCycle& c, const double* g, double* x, const PcgState* st, cudaStream_t s) {
  const int nc = c.nc, grid = vgrid(nc);
  double* d0 = c.work;
  double* d1 = c.work + nc;
  double* r = c.work + 2 * (size_t)nc;
  for (int cyc = 0; cyc < c.cycles; ++cyc) {
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 0 && cyc == 0) {  // pre-smoothing from x = 0: r = g
        k_cheb_first<<<grid, 256, 0, s>>>(g, c.dinv, c.cheb_c0, d0, x, r, nc, 0, st);
      } else {
        k_ell_resid<<<grid, 256, 0, s>>>(c.col, c.val, c.width, g, x, r, nc, st);
        k_cheb_first<<<grid, 256, 0, s>>>(r, c.dinv, c.cheb_c0, d0, x, nullptr, nc, 1, st);
      }
      double* dp = d0;
      double* dn = d1;
      for (int k = 1; k < c.deg; ++k) {
        k_cheb_step<<<grid, 256, 0, s>>>(c.col, c.val, c.width, c.dinv, dp, dn, r, x, c.cheb_a[k], c.cheb_b[k], nc,
                                         st);
        std::swap(dp, dn);
      }
      if (pass == 0) {  // aggregate correction of the residual
        k_ell_resid<<<grid, 256, 0, s>>>(c.col, c.val, c.width, g, x, r, nc, st);
        k_agg_restrict<<<vgrid(c.na), 256, 0, s>>>(c.aptr, c.amem, r, c.ga, c.na, st);
        k_dense_symv<<<std::min(152 * 8, (c.na + 7) / 8), 256, 0, s>>>(c.A00inv, c.ga, c.na, c.ya, st);
        k_agg_prolong<<<grid, 256, 0, s>>>(c.agg, c.ya, x, nc, st);
      }
    }
  }
  return cudaGetLastError();
}

int vcycle_launches(const CoarseCycle& c) { return c.cycles * (2 * c.deg + 6) - 1; }

}  // namespace sem
