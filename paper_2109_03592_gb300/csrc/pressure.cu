// Kernels of the staggered P_N - P_{N-2} pressure space (Sec. 2: velocity on
// the GLL points of order N, pressure on the Gauss-Legendre (GL) points of
// order N-2; Sec. 2, Eq. 5: the consistent Poisson equation for the pressure).
//
// With m = N - 1 GL points and n = N + 1 GLL points per direction, Ig[i][l] =
// l_l(zeta_i) (the GLL basis at the GL points) and DIg[i][l] = l_l'(zeta_i):
//   * factors F[b][a](q) = rho_i rho_j rho_k adj(J)_{ba} at every GL point q,
//     J = dx/dr of the isoparametric map (rho: GL weights, adj(J) = det(J) J^-1);
//   * weak divergence  (D u)_q = sum_{a,b} F[b][a](q) (C_b u_a)(q), where C_b
//     differentiates along direction b and interpolates along the other two
//     (DIg along b, Ig elsewhere);
//   * weak gradient    u_a = sum_b C_b^T (F[b][a] p), the transpose of D.
// The factors and the diagonal run one CTA per element in FP64; the weak
// gradient and divergence (pressure_line.cuh) apply each C_b as 1D
// contractions of whole lines held in registers, several elements per CTA,
// in FP64 or FP32.
#include "kernels.h"
#include "pressure_line.cuh"

namespace sem {

// GL-point factors.  Dynamic shared memory: X [3][n^3] (coordinates relative
// to the element's first node; D annihilates constants), Y and Yd [3][m][n][n]
// (the coordinates interpolated, resp. differentiated, along k).
__global__ void k_gl_factors(const double* __restrict__ xyz, const double* __restrict__ Ig,
                             const double* __restrict__ DIg, const double* __restrict__ rho, int n, int m, int64_t E,
                             double* __restrict__ F, int* bad) {
  extern __shared__ double sm[];
  const int n2 = n * n, n3 = n2 * n, m3 = m * m * m, mnn = m * n2;
  double* X = sm;
  double* Y = X + 3 * n3;
  double* Yd = Y + 3 * mnn;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  const double* xe = xyz + e * 3 * n3;
  for (int q = threadIdx.x; q < 3 * n3; q += blockDim.x) X[q] = xe[q] - xe[(q / n3) * n3];
  __syncthreads();
  // Y[c][kk][p][l] = sum_s Ig[kk][s] X[c][s][p][l], Yd likewise with DIg
  for (int q = threadIdx.x; q < 3 * mnn; q += blockDim.x) {
    const int c = q / mnn, r = q - c * mnn, kk = r / n2, pl = r - kk * n2;
    const double* Xc = X + c * n3 + pl;
    double a = 0.0, b = 0.0;
    for (int s = 0; s < n; ++s) {
      const double x = Xc[s * n2];
      a += Ig[kk * n + s] * x;
      b += DIg[kk * n + s] * x;
    }
    Y[q] = a;
    Yd[q] = b;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < m3; q += blockDim.x) {
    const int i = q % m, j = (q / m) % m, k = q / (m * m);
    double J[3][3];
    for (int c = 0; c < 3; ++c) {
      const double* Yc = Y + c * mnn + k * n2;
      const double* Ydc = Yd + c * mnn + k * n2;
      double dr = 0.0, ds = 0.0, dt = 0.0;
      for (int p = 0; p < n; ++p) {
        double ar = 0.0, as = 0.0, at = 0.0;
        for (int l = 0; l < n; ++l) {
          const double y = Yc[p * n + l], yd = Ydc[p * n + l];
          ar += DIg[i * n + l] * y;
          as += Ig[i * n + l] * y;
          at += Ig[i * n + l] * yd;
        }
        dr += Ig[j * n + p] * ar;
        ds += DIg[j * n + p] * as;
        dt += Ig[j * n + p] * at;
      }
      J[c][0] = dr;  // d x_c / d r
      J[c][1] = ds;  // d x_c / d s
      J[c][2] = dt;  // d x_c / d t
    }
    // cofactors C[a][b]; adj(J)[b][a] = C[a][b]
    double C[3][3];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    if (!(det > 0.0)) atomicExch(bad, 1);
    const double w = rho[i] * rho[j] * rho[k];
    double* Fe = F + e * 9 * m3 + q;
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) Fe[(3 * b + a) * m3] = w * C[a][b];
  }
}

// The weak gradient and divergence (k_pgrad_line, k_pdiv_line) are in
// pressure_line.cuh.

// ---- vector kernels of the pressure CG (pressure values, Euclidean products) ----
// Reductions are deterministic: block b sums its grid-stride slice in a fixed
// order and then a fixed shared-memory tree; k_psum_finish adds the block
// partials in index order.

static constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  return s[0];
}

// partial[block] = sum a_i b_i over the block's slice (b null: sum a_i)
__global__ void k_pdot(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* partial) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads)
    acc += b ? a[i] * b[i] : a[i];
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// w_i -= c; partial sums of p_i w_i
__global__ void k_pshift_dot(double* __restrict__ w, const double* __restrict__ p, double c, int64_t n,
                             double* partial) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const double v = w[i] - c;
    w[i] = v;
    acc += p[i] * v;
  }
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// y = a + beta y (the CG direction p = r + beta p)
__global__ void k_pdir(double* __restrict__ y, const double* __restrict__ a, double beta, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] + beta * y[i];
}

// r = g - c, p = r, x = 0; partial sums of r_i r_i
__global__ void k_pstart(const double* __restrict__ g, double c, double* __restrict__ r, double* __restrict__ p,
                         double* __restrict__ x, int64_t n, double* partial) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const double v = g[i] - c;
    r[i] = v;
    p[i] = v;
    x[i] = 0.0;
    acc += v * v;
  }
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_presidual_keep(const double* __restrict__ g, double cg, const double* __restrict__ w, double cw,
                                 double* __restrict__ r, int64_t n, double* partial) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const double v = (g[i] - cg) - (w[i] - cw);
    r[i] = v;
    acc += v * v;
  }
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[0] = sum of partial[0..cnt) (one CTA)
__global__ void k_psum_finish(const double* __restrict__ partial, int cnt, double* out) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < cnt; i += kRedThreads) acc += partial[i];
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) out[0] = t;
}

// ---- device-resident pressure CG (one PcgState; no host round trip per iteration) ----
// rho = <r, z>, rr = <r, r>, bb = ||Pm g||^2, pAp = sigma = <q, E q - mean>, aux = mean(E q),
// cz = mean(D^-1 r).  Every kernel returns at once when st->done.  Each reduction is a
// fixed per-block tree plus a fixed-order sum of the block partials by the last block.

// Sums of w, q w and q; the last block forms aux = mean(w), sigma = <q, w> - aux sum(q)
// (= <q, w - aux>), and alpha = rho / sigma (breakdown when sigma <= 0).
__global__ void k_pcg_psig(const double* __restrict__ q, const double* __restrict__ w, int64_t n, PcgState* st,
                           double* partial) {
  __shared__ double s[kRedThreads];
  __shared__ int sdone;
  if (threadIdx.x == 0) sdone = st->done;
  __syncthreads();
  if (sdone) return;
  double aw = 0.0, aqw = 0.0, aq = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const double wv = w[i], qv = q[i];
    aw += wv;
    aqw += qv * wv;
    aq += qv;
  }
  const double tw = block_sum(aw, s), tqw = block_sum(aqw, s), tq = block_sum(aq, s);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x] = tw;
    partial[3 * blockIdx.x + 1] = tqw;
    partial[3 * blockIdx.x + 2] = tq;
  }
  if (last_block(&st->cnt[0])) {
    double bw = 0.0, bqw = 0.0, bq = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kRedThreads) {
      bw += __ldcg(partial + 3 * b);
      bqw += __ldcg(partial + 3 * b + 1);
      bq += __ldcg(partial + 3 * b + 2);
    }
    const double sw = block_sum(bw, s), sqw = block_sum(bqw, s), sq = block_sum(bq, s);
    if (threadIdx.x == 0) {
      const double cw = sw / (double)n, sigma = sqw - cw * sq;
      st->aux = cw;
      st->pAp = sigma;
      if (!(sigma > 0.0)) {
        st->done = 1;
        st->status = 5;  // SEM_ERR_BREAKDOWN
      } else {
        st->alpha = st->rho / sigma;
      }
      st->cnt[0] = 0;
    }
  }
}

// x += alpha q; r -= alpha (w - aux); JAC: z = dinv r with its sum, <r, z> and sum(r).
// The last block forms rr, rho_new = <r, z - cz> (JAC) or rr, and applies the tests:
// rr <= tol2 bb (MIXED: gamma2 tol2 bb) pauses for the true residual (ru = 1); MIXED
// also pauses when rr <= delta2 rr_max at least `gap` iterations after the last
// replacement; maxit ends the run; otherwise beta = rho_new / rho.
template <bool JAC, bool MIXED>
__global__ void k_pcg_pupd(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ q,
                           const double* __restrict__ w, const double* __restrict__ dinv, double* __restrict__ z,
                           int64_t n, PcgState* st, double* partial, double gamma2, int gap) {
  __shared__ double s[kRedThreads];
  __shared__ int sdone;
  __shared__ double salpha, scw;
  if (threadIdx.x == 0) {
    sdone = st->done;
    salpha = st->alpha;
    scw = st->aux;
  }
  __syncthreads();
  if (sdone) return;
  const double alpha = salpha, cw = scw;
  double arr = 0.0, az = 0.0, arz = 0.0, ar = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    x[i] += alpha * q[i];
    const double v = r[i] - alpha * (w[i] - cw);
    r[i] = v;
    arr += v * v;
    if (JAC) {
      const double zv = dinv[i] * v;
      z[i] = zv;
      az += zv;
      arz += v * zv;
      ar += v;
    }
  }
  const double t0 = block_sum(arr, s);
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
  if (JAC) {
    t1 = block_sum(az, s);
    t2 = block_sum(arz, s);
    t3 = block_sum(ar, s);
  }
  if (threadIdx.x == 0) {
    partial[4 * blockIdx.x] = t0;
    partial[4 * blockIdx.x + 1] = t1;
    partial[4 * blockIdx.x + 2] = t2;
    partial[4 * blockIdx.x + 3] = t3;
  }
  if (last_block(&st->cnt[1])) {
    double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kRedThreads) {
      b0 += __ldcg(partial + 4 * b);
      b1 += __ldcg(partial + 4 * b + 1);
      b2 += __ldcg(partial + 4 * b + 2);
      b3 += __ldcg(partial + 4 * b + 3);
    }
    const double rr = block_sum(b0, s);
    double sz = 0.0, srz = 0.0, sr = 0.0;
    if (JAC) {
      sz = block_sum(b1, s);
      srz = block_sum(b2, s);
      sr = block_sum(b3, s);
    }
    if (threadIdx.x == 0) {
      const double cz = JAC ? sz / (double)n : 0.0;
      const double rho_new = JAC ? srz - cz * sr : rr;
      st->iter += 1;
      st->rr = rr;
      st->cz = cz;
      if (rr != rr || rho_new != rho_new) {
        st->done = 1;
        st->status = 5;
      } else if (rr <= (MIXED ? gamma2 : 1.0) * st->tol2 * st->bb) {
        st->done = 1;
        st->ru = 1;  // the host checks the true residual
      } else if (MIXED && rr <= st->delta2 * st->rr_max && st->iter - st->last >= gap) {
        st->done = 1;
        st->ru = 1;  // reliable update
      } else if (st->iter >= st->maxit) {
        st->done = 1;
        st->status = 4;  // SEM_ERR_NOT_CONVERGED
      } else {
        if (rr > st->rr_max) st->rr_max = rr;
        st->beta = rho_new / st->rho;
        st->rho = rho_new;
      }
      st->cnt[1] = 0;
    }
  }
}

// q = (zd - cz) + beta q (zd = z with Jacobi, r without, where cz = 0)
__global__ void k_pcg_pdir(double* __restrict__ q, const double* __restrict__ zd, int64_t n,
                           const PcgState* __restrict__ st) {
  if (st->done) return;
  const double beta = st->beta, cz = st->cz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = (zd[i] - cz) + beta * q[i];
}

// FP32 copies for the mixed-precision pressure solve
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void k_recip_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)(1.0 / a[i]);
}

// r = (g - cg) - (w - cw) (the true residual Pm (g - E x)); partial sums of r_i r_i
__global__ void k_presidual_keep(const double* __restrict__ g, double cg, const double* __restrict__ w, double cw,
                                 double* __restrict__ r, int64_t n, double* partial);

// diag(E) (recip = 0) or its reciprocal, one CTA per element.  Unit pressure q gives
// D_a^T e_q = the row D_a[q, :] on the element's GLL points, which QQ^T leaves
// as it is at the element's own copies (no element holds two copies of one
// node), so E_qq = sum_a sum_l D_a[q, l]^2 wgt_l with wgt = mask / (QQ^T B).
// With D_a[q, l] = sum_b F[b][a](q) C_b[q, l]:
//   E_qq = sum_a sum_{b, b'} F[b][a](q) F[b'][a](q) S_{bb'}(q),
//   S_{bb'}(q) = sum_l C_b[q, l] C_b'[q, l] wgt_l,
// and S_{bb'} is a sum factorisation with the 1D matrices Ig*Ig, Ig*DIg or
// DIg*DIg (elementwise) along each direction, by how many of b, b' are that
// direction.  Shared memory: X [3][m][n], wgt [n^3], T1 [n][n][m],
// T2 [n][m][m], S [6][m^3].
__global__ void k_pdiag(const double* __restrict__ F, const double* __restrict__ Ig, const double* __restrict__ DIg,
                        const uint8_t* __restrict__ wm, const double* __restrict__ dB, int n, int m, int64_t E,
                        double* __restrict__ out, int recip) {
  extern __shared__ double sm[];
  const int n2 = n * n, n3 = n2 * n, m2 = m * m, m3 = m2 * m, mn = m * n;
  double* X = sm;
  double* wgt = X + 3 * mn;
  double* T1 = wgt + n3;
  double* T2 = T1 + n2 * m;
  double* S = T2 + n * m2;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  for (int q = threadIdx.x; q < mn; q += blockDim.x) {
    X[q] = Ig[q] * Ig[q];
    X[mn + q] = Ig[q] * DIg[q];
    X[2 * mn + q] = DIg[q] * DIg[q];
  }
  for (int q = threadIdx.x; q < n3; q += blockDim.x) {
    const int64_t l = e * n3 + q;
    wgt[q] = (wm[l] & 0x80) ? 0.0 : 1.0 / dB[l];
  }
  __syncthreads();
  const int pb[6] = {0, 1, 2, 0, 0, 1}, pc[6] = {0, 1, 2, 1, 2, 2};
  for (int c = 0; c < 6; ++c) {
    const int b = pb[c], b2 = pc[c];
    const double* Xi = X + ((b == 0) + (b2 == 0)) * mn;
    const double* Xj = X + ((b == 1) + (b2 == 1)) * mn;
    const double* Xk = X + ((b == 2) + (b2 == 2)) * mn;
    // T1[k][j][I] = sum_i Xi[I][i] wgt[k][j][i]
    for (int q = threadIdx.x; q < n2 * m; q += blockDim.x) {
      const int I = q % m, kj = q / m;
      double a = 0.0;
      for (int i = 0; i < n; ++i) a += Xi[I * n + i] * wgt[kj * n + i];
      T1[q] = a;
    }
    __syncthreads();
    // T2[k][J][I] = sum_j Xj[J][j] T1[k][j][I]
    for (int q = threadIdx.x; q < n * m2; q += blockDim.x) {
      const int I = q % m, J = (q / m) % m, k = q / m2;
      double a = 0.0;
      for (int j = 0; j < n; ++j) a += Xj[J * n + j] * T1[(k * n + j) * m + I];
      T2[q] = a;
    }
    __syncthreads();
    // S_c[K][J][I] = sum_k Xk[K][k] T2[k][J][I]
    for (int q = threadIdx.x; q < m3; q += blockDim.x) {
      const int JI = q % m2, K = q / m2;
      double a = 0.0;
      for (int k = 0; k < n; ++k) a += Xk[K * n + k] * T2[k * m2 + JI];
      S[c * m3 + q] = a;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < m3; q += blockDim.x) {
    const double* Fe = F + e * 9 * m3 + q;
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double f0 = Fe[(0 + a) * m3], f1 = Fe[(3 + a) * m3], f2 = Fe[(6 + a) * m3];
      d += f0 * f0 * S[q] + f1 * f1 * S[m3 + q] + f2 * f2 * S[2 * m3 + q] +
           2.0 * (f0 * f1 * S[3 * m3 + q] + f0 * f2 * S[4 * m3 + q] + f1 * f2 * S[5 * m3 + q]);
    }
    out[e * m3 + q] = recip ? (d > 0.0 ? 1.0 / d : 0.0) : d;
  }
}

// z = dinv * r; partial sums of z_i (its mean is removed by k_pshift_dot)
__global__ void k_pscale(const double* __restrict__ r, const double* __restrict__ dinv, double* __restrict__ z,
                         int64_t n, double* partial) {
  __shared__ double s[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const double v = dinv[i] * r[i];
    z[i] = v;
    acc += v;
  }
  const double t = block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// ---- launchers ---------------------------------------------------------------

static constexpr int kPressureThreads = 256;
static constexpr int kPressureRedBlocks = 2 * 152;  // reduction grid: two CTAs per SM

size_t gl_factors_smem(int n, int m) { return sizeof(double) * (3 * n * n * n + 6 * m * n * n); }
cudaError_t launch_gl_factors(const double* xyz, const double* Ig, const double* DIg, const double* rho, int n, int m,
                              int64_t E, double* F, int* bad, cudaStream_t s) {
  const size_t smem = gl_factors_smem(n, m);
  cudaError_t err = cudaFuncSetAttribute(k_gl_factors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_gl_factors<<<(unsigned)E, kPressureThreads, smem, s>>>(xyz, Ig, DIg, rho, n, m, E, F, bad);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_pgrad_n(const T* p, const T* F, const T* Ig, const T* DIg, int64_t E, T* u, int64_t n_local,
                           cudaStream_t s) {
  using S = pline::Shape<T, N>;
  static DeviceOnce once;
  cudaError_t err = once.get([&](int, int*) {
    return cudaFuncSetAttribute(pline::k_pgrad_line<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
  });
  if (err != cudaSuccess) return err;
  if (E == 0) return cudaSuccess;
  pline::k_pgrad_line<T, N><<<(unsigned)((E + S::EPB - 1) / S::EPB), pline::kThreads, S::smem, s>>>(p, F, Ig, DIg, E,
                                                                                                  u, n_local);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t launch_pdiv_n(const T* u, const T* dB, const T* invB, const T* F, const T* Ig, const T* DIg, int64_t E,
                          T* out, int64_t n_local, cudaStream_t s) {
  using S = pline::Shape<T, N>;
  static DeviceOnce once;
  cudaError_t err = once.get([&](int, int*) {
    return cudaFuncSetAttribute(pline::k_pdiv_line<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
  });
  if (err != cudaSuccess) return err;
  if (E == 0) return cudaSuccess;
  pline::k_pdiv_line<T, N><<<(unsigned)((E + S::EPB - 1) / S::EPB), pline::kThreads, S::smem, s>>>(
      u, dB, invB, F, Ig, DIg, E, out, n_local);
  return cudaGetLastError();
}

#define SEM_PRESSURE_ORDERS(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

template <typename T>
cudaError_t launch_pgrad(const T* p, const T* F, const T* Ig, const T* DIg, int n, int m, int64_t E, T* u,
                         int64_t n_local, cudaStream_t s) {
  if (m != n - 2) return cudaErrorInvalidValue;
  switch (n - 1) {
#define SEM_CASE(N) \
  case N:           \
    return launch_pgrad_n<T, N>(p, F, Ig, DIg, E, u, n_local, s);
    SEM_PRESSURE_ORDERS(SEM_CASE)
#undef SEM_CASE
    default: return cudaErrorNotSupported;
  }
}
template cudaError_t launch_pgrad<double>(const double*, const double*, const double*, const double*, int, int, int64_t,
                                          double*, int64_t, cudaStream_t);
template cudaError_t launch_pgrad<float>(const float*, const float*, const float*, const float*, int, int, int64_t,
                                         float*, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_pdiv(const T* u, const T* dB, const T* invB, const T* F, const T* Ig, const T* DIg, int n, int m,
                        int64_t E, T* out, int64_t n_local, cudaStream_t s) {
  if (m != n - 2) return cudaErrorInvalidValue;
  switch (n - 1) {
#define SEM_CASE(N) \
  case N:           \
    return launch_pdiv_n<T, N>(u, dB, invB, F, Ig, DIg, E, out, n_local, s);
    SEM_PRESSURE_ORDERS(SEM_CASE)
#undef SEM_CASE
    default: return cudaErrorNotSupported;
  }
}
template cudaError_t launch_pdiv<double>(const double*, const double*, const double*, const double*, const double*,
                                         const double*, int, int, int64_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_pdiv<float>(const float*, const float*, const float*, const float*, const float*,
                                        const float*, int, int, int64_t, float*, int64_t, cudaStream_t);

void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  k_to_f32<<<kPressureRedBlocks, kRedThreads, 0, s>>>(a, b, n);
}
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  k_to_f64<<<kPressureRedBlocks, kRedThreads, 0, s>>>(a, b, n);
}
void launch_recip_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  k_recip_f32<<<kPressureRedBlocks, kRedThreads, 0, s>>>(a, b, n);
}

int pressure_red_blocks() { return kPressureRedBlocks; }

cudaError_t launch_pdot(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s) {
  k_pdot<<<kPressureRedBlocks, kRedThreads, 0, s>>>(a, b, n, partial);
  k_psum_finish<<<1, kRedThreads, 0, s>>>(partial, kPressureRedBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_pdiag(const double* F, const double* Ig, const double* DIg, const uint8_t* wm, const double* dB,
                        int n, int m, int64_t E, double* out, int recip, cudaStream_t s) {
  const size_t smem = sizeof(double) * (3 * m * n + n * n * n + n * n * m + n * m * m + 6 * m * m * m);
  cudaError_t err = cudaFuncSetAttribute(k_pdiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E == 0) return cudaSuccess;
  k_pdiag<<<(unsigned)E, kPressureThreads, smem, s>>>(F, Ig, DIg, wm, dB, n, m, E, out, recip);
  return cudaGetLastError();
}

cudaError_t launch_pscale(const double* r, const double* dinv, double* z, int64_t n, double* partial, double* out,
                          cudaStream_t s) {
  k_pscale<<<kPressureRedBlocks, kRedThreads, 0, s>>>(r, dinv, z, n, partial);
  k_psum_finish<<<1, kRedThreads, 0, s>>>(partial, kPressureRedBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_pshift_dot(double* w, const double* p, double c, int64_t n, double* partial, double* out,
                              cudaStream_t s) {
  k_pshift_dot<<<kPressureRedBlocks, kRedThreads, 0, s>>>(w, p, c, n, partial);
  k_psum_finish<<<1, kRedThreads, 0, s>>>(partial, kPressureRedBlocks, out);
  return cudaGetLastError();
}


cudaError_t launch_pdir(double* y, const double* a, double beta, int64_t n, cudaStream_t s) {
  k_pdir<<<kPressureRedBlocks, kRedThreads, 0, s>>>(y, a, beta, n);
  return cudaGetLastError();
}

cudaError_t launch_pstart(const double* g, double c, double* r, double* p, double* x, int64_t n, double* partial,
                          double* out, cudaStream_t s) {
  k_pstart<<<kPressureRedBlocks, kRedThreads, 0, s>>>(g, c, r, p, x, n, partial);
  k_psum_finish<<<1, kRedThreads, 0, s>>>(partial, kPressureRedBlocks, out);
  return cudaGetLastError();
}


cudaError_t launch_pcg_psig(const double* q, const double* w, int64_t n, PcgState* st, double* partial,
                            cudaStream_t s) {
  k_pcg_psig<<<kPressureRedBlocks, kRedThreads, 0, s>>>(q, w, n, st, partial);
  return cudaGetLastError();
}

cudaError_t launch_pcg_pupd(bool jac, bool mixed, double* x, double* r, const double* q, const double* w,
                            const double* dinv, double* z, int64_t n, PcgState* st, double* partial, double gamma2,
                            int gap, cudaStream_t s) {
  if (jac && mixed)
    k_pcg_pupd<true, true><<<kPressureRedBlocks, kRedThreads, 0, s>>>(x, r, q, w, dinv, z, n, st, partial, gamma2, gap);
  else if (jac)
    k_pcg_pupd<true, false><<<kPressureRedBlocks, kRedThreads, 0, s>>>(x, r, q, w, dinv, z, n, st, partial, gamma2, gap);
  else if (mixed)
    k_pcg_pupd<false, true><<<kPressureRedBlocks, kRedThreads, 0, s>>>(x, r, q, w, dinv, z, n, st, partial, gamma2, gap);
  else
    k_pcg_pupd<false, false><<<kPressureRedBlocks, kRedThreads, 0, s>>>(x, r, q, w, dinv, z, n, st, partial, gamma2,
                                                                       gap);
  return cudaGetLastError();
}

cudaError_t launch_pcg_pdir(double* q, const double* zd, int64_t n, const PcgState* st, cudaStream_t s) {
  k_pcg_pdir<<<kPressureRedBlocks, kRedThreads, 0, s>>>(q, zd, n, st);
  return cudaGetLastError();
}

int pressure_partials() { return 4 * kPressureRedBlocks; }

cudaError_t launch_presidual_keep(const double* g, double cg, const double* w, double cw, double* r, int64_t n,
                                  double* partial, double* out, cudaStream_t s) {
  k_presidual_keep<<<kPressureRedBlocks, kRedThreads, 0, s>>>(g, cg, w, cw, r, n, partial);
  k_psum_finish<<<1, kRedThreads, 0, s>>>(partial, kPressureRedBlocks, out);
  return cudaGetLastError();
}

}  // namespace sem
