// Mesh set-up kernels: GLL point coordinates of the built-in meshes, the
// geometric factors g1..g6 and mass B used by Alg. 1, the local diagonal of
// the stiffness (for the Jacobi preconditioner) and precision conversions.
//
// Geometry (the paper uses g1xyz..g6xyz without defining them; the standard
// isoparametric reading): J_ab = dx_a/dr_b from D applied to the nodal
// coordinates, G = w_i w_j w_k det(J) J^{-1} J^{-T} with g1..g6 = G_rr, G_ss,
// G_tt, G_rs, G_rt, G_st, and B = w_i w_j w_k det(J).
#include "kernels.h"

namespace sem {

__device__ __forceinline__ double lerp_ends(double a, double b, double xi) {
  return a * (1.0 - xi) * 0.5 + b * (1.0 + xi) * 0.5;  // exact at xi = -1 and xi = +1
}

// One thread per GLL point.  Box element e = ex + nx (ey + ny ez).
__global__ void k_coords_box(double* xyz, const double* __restrict__ xi, int n, int64_t E, int nx, int ny,
                             int nz, double lx, double ly, double lz) {
  const int64_t n3 = (int64_t)n * n * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E * n3; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / n3;
    const int p = (int)(q % n3), i = p % n, j = (p / n) % n, k = p / (n * n);
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    double* out = xyz + e * 3 * n3 + p;
    out[0] = lerp_ends(lx * ex / nx, lx * (ex + 1) / nx, xi[i]);
    out[n3] = lerp_ends(ly * ey / ny, ly * (ey + 1) / ny, xi[j]);
    out[2 * n3] = lerp_ends(lz * ez / nz, lz * (ez + 1) / nz, xi[k]);
  }
}

// O-grid pipe (see sem_mesh_desc for the map and the element order).
__global__ void k_coords_pipe(double* xyz, const double* __restrict__ xi, const double* __restrict__ tlev, int n,
                              int64_t E, int nc, int nr, int nzp, double R, double L, double a) {
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t n2d = (int64_t)nc * (nc + 4 * nr);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E * n3; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / n3;
    const int p = (int)(q % n3), i = p % n, j = (p / n) % n, k = p / (n * n);
    const int64_t layer = e / n2d, e2 = e % n2d;
    double x, y;
    if (e2 < (int64_t)nc * nc) {
      const int ex = (int)(e2 % nc), ey = (int)(e2 / nc);
      x = lerp_ends(-a + 2.0 * a * ex / nc, -a + 2.0 * a * (ex + 1) / nc, xi[i]);
      y = lerp_ends(-a + 2.0 * a * ey / nc, -a + 2.0 * a * (ey + 1) / nc, xi[j]);
    } else {
      const int64_t rest = e2 - (int64_t)nc * nc;
      const int qb = (int)(rest / ((int64_t)nc * nr));
      const int r = (int)((rest % ((int64_t)nc * nr)) / nc), m = (int)(rest % nc);
      const double t = lerp_ends(tlev[r], tlev[r + 1], xi[i]);
      const double s = lerp_ends(-1.0 + 2.0 * m / nc, -1.0 + 2.0 * (m + 1) / nc, xi[j]);
      const double th = s * M_PI / 4.0;
      const double px = (1.0 - t) * a + t * R * cos(th);
      const double py = (1.0 - t) * a * s + t * R * sin(th);
      switch (qb) {
        case 0: x = px; y = py; break;
        case 1: x = -py; y = px; break;
        case 2: x = -px; y = -py; break;
        default: x = py; y = -px; break;
      }
    }
    double* out = xyz + e * 3 * n3 + p;
    out[0] = x;
    out[n3] = y;
    out[2 * n3] = lerp_ends(L * layer / nzp, L * (layer + 1) / nzp, xi[k]);
  }
}

// One block per element; threads loop over the element's points.
// Dynamic shared memory: 3 n^3 doubles (the coordinates).
__global__ void k_geometry(const double* __restrict__ xyz, double* __restrict__ G, double* __restrict__ B,
                           const double* __restrict__ Dg, const double* __restrict__ wg, int n, int64_t E,
                           int* bad) {
  extern __shared__ double sx[];
  const int n3 = n * n * n;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  // coordinates relative to the element's first node: D annihilates constants,
  // and this avoids cancelling O(|x|) terms into an O(h) derivative
  for (int q = threadIdx.x; q < 3 * n3; q += blockDim.x) sx[q] = xyz[e * 3 * n3 + q] - xyz[e * 3 * n3 + (q / n3) * n3];
  __syncthreads();
  for (int p = threadIdx.x; p < n3; p += blockDim.x) {
    const int i = p % n, j = (p / n) % n, k = p / (n * n);
    double J[3][3];
    for (int c = 0; c < 3; ++c) {
      const double* X = sx + c * n3;
      double dr = 0.0, ds = 0.0, dt = 0.0;
      for (int l = 0; l < n; ++l) {
        dr += Dg[i * n + l] * X[l + n * (j + n * k)];
        ds += Dg[j * n + l] * X[i + n * (l + n * k)];
        dt += Dg[k * n + l] * X[i + n * (j + n * l)];
      }
      J[c][0] = dr;
      J[c][1] = ds;
      J[c][2] = dt;
    }
    // cofactors: adj(J)[b][a] = C[a][b]; J^{-1} = adj(J) / det(J)
    const double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const double C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const double C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const double C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const double C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
    if (!(det > 0.0)) atomicExch(bad, 1);
    // Jinv[b][a] = d r_b / d x_a = C[a][b] / det.  G = w3 det Jinv Jinv^T = w3 / det * C^T C
    const double w3 = wg[i] * wg[j] * wg[k];
    const double s = w3 / det;
    const double g1 = s * (C00 * C00 + C10 * C10 + C20 * C20);
    const double g2 = s * (C01 * C01 + C11 * C11 + C21 * C21);
    const double g3 = s * (C02 * C02 + C12 * C12 + C22 * C22);
    const double g4 = s * (C00 * C01 + C10 * C11 + C20 * C21);
    const double g5 = s * (C00 * C02 + C10 * C12 + C20 * C22);
    const double g6 = s * (C01 * C02 + C11 * C12 + C21 * C22);
    double* Ge = G + e * 6 * n3 + p;
    Ge[0] = g1;
    Ge[n3] = g2;
    Ge[2 * n3] = g3;
    Ge[3 * n3] = g4;
    Ge[4 * n3] = g5;
    Ge[5 * n3] = g6;
    B[e * n3 + p] = w3 * det;
  }
}

// Local diagonal of the stiffness part of A_L (h1 = 1, h2 = 0):
// sum_l D_li^2 g1_ljk + sum_l D_lj^2 g2_ilk + sum_l D_lk^2 g3_ijl
// + 2 D_ii D_jj g4 + 2 D_ii D_kk g5 + 2 D_jj D_kk g6.
__global__ void k_local_diag(const double* __restrict__ G, double* __restrict__ dK, const double* __restrict__ Dg,
                             int n, int64_t E) {
  const int64_t n3 = (int64_t)n * n * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E * n3; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / n3;
    const int p = (int)(q % n3), i = p % n, j = (p / n) % n, k = p / (n * n);
    const double* Ge = G + e * 6 * n3;
    double s = 0.0;
    for (int l = 0; l < n; ++l) {
      const double a = Dg[l * n + i], b = Dg[l * n + j], c = Dg[l * n + k];
      s += a * a * Ge[l + n * (j + n * k)];
      s += b * b * Ge[n3 + i + n * (l + n * k)];
      s += c * c * Ge[2 * n3 + i + n * (j + n * l)];
    }
    const double di = Dg[i * n + i], dj = Dg[j * n + j], dk = Dg[k * n + k];
    s += 2.0 * di * dj * Ge[3 * n3 + p] + 2.0 * di * dk * Ge[4 * n3 + p] + 2.0 * dj * dk * Ge[5 * n3 + p];
    dK[q] = s;
  }
}

// hi = round-to-nearest float(v), lo = float(v - hi): v ~ hi + lo to ~2^-48 relative.
__global__ void k_split_f64(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo, int64_t m) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[q];
    const float h = __double2float_rn(x);
    hi[q] = h;
    if (lo) lo[q] = __double2float_rn(x - (double)h);
  }
}

// Per-point coefficients folded into the stored factors: cG = h1[q] G (all six
// factors of the point) and cB = h2[q] B.  Alg. 1 scales (G . grad u) at each
// point by h1 of that point, which is h1 G at the point; the mass term scales
// B u by h2.  Bit 0 / 1 of *bad flags an h1 <= 0 / h2 < 0 or a non-finite
// value.
__global__ void k_fold_coef(const double* __restrict__ G, const double* __restrict__ B, const double* __restrict__ h1,
                            const double* __restrict__ h2, double* __restrict__ cG, double* __restrict__ cB, int n3,
                            int64_t P, int* bad) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / n3, r = q - e * n3;
    if (h1) {
      const double c = h1[q];
      if (!(c > 0.0) || !isfinite(c)) atomicOr(bad, 1);
      for (int k = 0; k < 6; ++k) cG[(e * 6 + k) * n3 + r] = c * G[(e * 6 + k) * n3 + r];
    }
    if (h2) {
      const double c = h2[q];
      if (!(c >= 0.0) || !isfinite(c)) atomicOr(bad, 2);
      cB[q] = c * B[q];
    }
  }
}

__global__ void k_weights(const uint8_t* __restrict__ wm, double* mult, double* mask, int64_t m) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t b = wm[q];
    if (mult) mult[q] = (double)(b & 0x7f);
    if (mask) mask[q] = (b & 0x80) ? 0.0 : 1.0;
  }
}

// ---- launchers ---------------------------------------------------------------

static int grid_for(int64_t m, int threads) {
  int64_t g = (m + threads - 1) / threads;
  const int64_t cap = 152LL * 32;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

void launch_coords_box(double* xyz, const double* xi, int n, int64_t E, int nx, int ny, int nz, double lx,
                       double ly, double lz, cudaStream_t s) {
  k_coords_box<<<grid_for(E * n * n * n, 256), 256, 0, s>>>(xyz, xi, n, E, nx, ny, nz, lx, ly, lz);
}

void launch_coords_pipe(double* xyz, const double* xi, const double* tlev, int n, int64_t E, int nc, int nr,
                        int nzp, double R, double L, double a, cudaStream_t s) {
  k_coords_pipe<<<grid_for(E * n * n * n, 256), 256, 0, s>>>(xyz, xi, tlev, n, E, nc, nr, nzp, R, L, a);
}

cudaError_t launch_geometry(const double* xyz, double* G, double* B, const double* D, const double* w, int n,
                            int64_t E, int* bad, cudaStream_t s) {
  const size_t smem = 3 * sizeof(double) * n * n * n;
  cudaError_t err = cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // grid dimension x may hold up to 2^31 - 1 blocks
  k_geometry<<<(unsigned)E, 256, smem, s>>>(xyz, G, B, D, w, n, E, bad);
  return cudaGetLastError();
}

void launch_local_diag(const double* G, double* dK, const double* D, int n, int64_t E, cudaStream_t s) {
  k_local_diag<<<grid_for(E * n * n * n, 256), 256, 0, s>>>(G, dK, D, n, E);
}

void launch_split_f64(const double* v, float* hi, float* lo, int64_t m, cudaStream_t s) {
  k_split_f64<<<grid_for(m, 256), 256, 0, s>>>(v, hi, lo, m);
}

void launch_fold_coef(const double* G, const double* B, const double* h1, const double* h2, double* cG, double* cB,
                      int n, int64_t P, int* bad, cudaStream_t s) {
  k_fold_coef<<<grid_for(P, 256), 256, 0, s>>>(G, B, h1, h2, cG, cB, n * n * n, P, bad);
}

void launch_weights(const uint8_t* wm, double* mult, double* mask, int64_t m, cudaStream_t s) {
  k_weights<<<grid_for(m, 256), 256, 0, s>>>(wm, mult, mask, m);
}

}  // namespace sem
