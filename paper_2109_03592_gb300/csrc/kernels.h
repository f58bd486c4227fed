// Kernel launchers and their parameter blocks.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_util.cuh"
#include "launch_once.h"

namespace sem {

// Host-side tally of kernel launches issued by the library (sem_kernel_launches).
void count_launches(uint64_t n);

// ---- mesh set-up (geom.cu) ----
void launch_coords_box(double* xyz, const double* xi, int n, int64_t E, int nx, int ny, int nz, double lx,
                       double ly, double lz, cudaStream_t s);
void launch_coords_pipe(double* xyz, const double* xi, const double* tlev, int n, int64_t E, int nc, int nr,
                        int nzp, double R, double L, double a, cudaStream_t s);
cudaError_t launch_geometry(const double* xyz, double* G, double* B, const double* D, const double* w, int n,
                            int64_t E, int* bad, cudaStream_t s);
void launch_local_diag(const double* G, double* dK, const double* D, int n, int64_t E, cudaStream_t s);
void launch_fold_coef(const double* G, const double* B, const double* h1, const double* h2, double* cG, double* cB,
                      int n, int64_t P, int* bad, cudaStream_t s);
void launch_split_f64(const double* v, float* hi, float* lo, int64_t m, cudaStream_t s);
void launch_weights(const uint8_t* wm, double* mult, double* mask, int64_t m, cudaStream_t s);

// ---- local operator (ax_*.cu) ----
template <typename T>
struct AxParams {
  const T* u;        // input (plain variant)
  T* w;              // output A_L u
  const T* G;        // [E][6][n3]
  const T* B;        // [E][n3] (Helmholtz term)
  const T* D;        // [n*n]
  T h1, h2;
  int helm;          // h2 != 0
  int64_t E;
  // fused-PCG variant: p <- z + beta p, u := p, partial <p, A_L p>
  const T* z;
  T* p;
  PcgState* st;
  double* partial;   // [gridDim.x]
  int* err;          // device error word (bounded-wait timeouts of the bulk-copy kernels)
  T* pout = nullptr;  // fused: the new direction goes here (nullptr: over p)
};

// Double-float (FP32 pair) FP64-accurate variant: G = Ghi + Glo, D = Dhi + Dlo,
// u and w FP64 in memory.
struct AxDFParams {
  const double* u;
  double* w;
  const float* Ghi;
  const float* Glo;
  const float* Bhi;  // B = Bhi + Blo (Helmholtz term)
  const float* Blo;
  const float* Dhi;
  const float* Dlo;
  double h1, h2;
  int helm;
  int64_t E;
  const double* z;
  double* p;
  PcgState* st;
  double* partial;
  const double* eo64;  // even-odd coefficient tables (even n; see sem_mesh::eo64)
  const float* eodf;
  double* pout = nullptr;  // fused: the new direction goes here (nullptr: over p)
};

// Kernel variants of the local operator for one (N, precision): 0 and 1 are
// the register/shared-memory kernels with ~256 / ~128 threads per CTA; 2 and
// 3 (FP32, even n only) the persistent bulk-copy pipelined kernels with
// ~128 threads x 3 stages / ~256 threads x 2 stages; for the double-float
// FP64 operator 2 and 3 are the even-odd kernels (even n only).  A launch of a variant
// that does not exist for (N, precision) returns cudaErrorNotSupported.
int ax_num_variants();
int ax_elems_per_block(int N, int variant);
cudaError_t launch_ax_f64(int N, int variant, bool fused, const AxParams<double>& p, cudaStream_t s, int* grid_out);
cudaError_t launch_ax_f32(int N, int variant, bool fused, const AxParams<float>& p, cudaStream_t s, int* grid_out);
cudaError_t launch_ax_df(int N, int variant, bool fused, const AxDFParams& p, cudaStream_t s, int* grid_out);
int ax_df_available(int N);

// ---- gather-scatter (gs.cu) ----
// Device view of the class-based plan (see GsPlan in sem_internal.h).
struct GsDev {
  const int32_t* idx;
  const int32_t* gptr;
  int64_t off[9];
  int64_t cnt[9];
  const int4* units;  // {class, first node, count, 0} in processing order
  int64_t nunits;
};
template <typename T>
cudaError_t launch_gs(T* v, const GsDev& g, int apply_mask, const PcgState* st, cudaStream_t s);

// ---- PCG vector kernels (pcg.cu) ----
template <typename T>
struct VecParams {
  T* x;
  T* r;
  T* z;
  T* p;
  const T* w;
  const T* minv;
  const T* b;
  const uint8_t* wm;
  int64_t n;
  PcgState* st;
  double* partial;  // [3 * grid]
  const T* p2 = nullptr;  // the previous direction (x updated with two directions, see k_pcg_update)
};
int vec_grid();
// ext = true: an external preconditioner (its kernels write z = M^{-1} r
// between k_pcg_update and launch_pcg_rho; init and restart read that z).
// xmode: 0 x += alpha p; 1 x not updated (alpha kept as alpha_prev, xpend
// set); 2 x += alpha_prev p2 + alpha p.
template <typename T>
cudaError_t launch_pcg_update(const VecParams<T>& p, cudaStream_t s, bool ext = false, int xmode = 0);
// Completes a pair of x updates after a pause (k_pcg_update xmode 1 was the
// last): x += alpha_prev p2, p = p2; clears xpend.
template <typename T>
cudaError_t launch_pcg_xflush(T* x, T* p, const T* p2, PcgState* st, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_pcg_init(const VecParams<T>& p, cudaStream_t s, bool ext = false);
template <typename T>
cudaError_t launch_pcg_restart(const VecParams<T>& p, cudaStream_t s, bool ext = false);
// rho_new = <r, z>_W, beta = rho_new / rho (skipped once st->done); with
// zout, z (type Z) holds M^{-1} (zscale r) and zout = z / zscale is written.
template <typename T, typename Z>
cudaError_t launch_pcg_rho(const T* r, const Z* z, T* zout, double zscale, const uint8_t* wm, int64_t n, PcgState* st,
                           double* partial, cudaStream_t s);
void launch_set_bb(PcgState* st, double bb, double delta2, cudaStream_t s);

void launch_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t s);
void launch_mask(double* x, const uint8_t* wm, int64_t n, cudaStream_t s);
void launch_minv(double* minv, float* minv32, const double* dK, const double* dB, const uint8_t* wm, double h1,
                 double h2, int64_t n, cudaStream_t s);
// r = b - w, st->aux = <r, r>_W, st->bb = <b, b>_W (when set_bb)
cudaError_t launch_residual(double* r, const double* b, const double* w, const uint8_t* wm, int64_t n, PcgState* st,
                            double* partial, int set_bb, cudaStream_t s);
// r32 = float(sc * r)
void launch_scale_to_f32(float* r32, const double* r, double sc, int64_t n, cudaStream_t s);
// x += sc * double(d32)
void launch_accumulate(double* x, const float* d32, double sc, int64_t n, cudaStream_t s);
void launch_zero_f32(float* a, int64_t n, cudaStream_t s);
// pAp and alpha from the per-block partials of a fused local operator
cudaError_t launch_pap_finish(const double* partial, int count, PcgState* st, cudaStream_t s);

// ---- P_N - P_{N-2} pressure space (pressure.cu) ----
// m = N - 1 GL points, n = N + 1 GLL points per direction; Ig, DIg [m][n];
// F [E][9][m^3] (index 3 b + a); u [3][n_local]; pressures [E][m^3].
size_t gl_factors_smem(int n, int m);
cudaError_t launch_gl_factors(const double* xyz, const double* Ig, const double* DIg, const double* rho, int n, int m,
                              int64_t E, double* F, int* bad, cudaStream_t s);
// T = double, or float for the FP32 operator (factors and basis rounded from FP64)
template <typename T>
cudaError_t launch_pgrad(const T* p, const T* F, const T* Ig, const T* DIg, int n, int m, int64_t E, T* u,
                         int64_t n_local, cudaStream_t s);
// v_a = u_a / dB (dB given), u_a invB (invB given), or u_a
template <typename T>
cudaError_t launch_pdiv(const T* u, const T* dB, const T* invB, const T* F, const T* Ig, const T* DIg, int n, int m,
                        int64_t E, T* out, int64_t n_local, cudaStream_t s);
void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
void launch_recip_f32(const double* a, float* b, int64_t n, cudaStream_t s);
// r = (g - cg) - (w - cw), out[0] = <r, r>
cudaError_t launch_presidual_keep(const double* g, double cg, const double* w, double cw, double* r, int64_t n,
                                  double* partial, double* out, cudaStream_t s);
// Pressure-CG vector kernels; each reduction writes its (deterministic) sum to
// out[0] on the device, using partial[pressure_red_blocks()] as scratch.
int pressure_red_blocks();
cudaError_t launch_pdot(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s);
// out [E m^3] = diag(E), or 1 / diag(E) with recip (the pressure operator's
// diagonal; wm's Dirichlet bit is the velocity mask, dB the assembled mass)
cudaError_t launch_pdiag(const double* F, const double* Ig, const double* DIg, const uint8_t* wm, const double* dB,
                        int n, int m, int64_t E, double* out, int recip, cudaStream_t s);
// Device-resident pressure CG steps (state in a PcgState, see pressure.cu):
// sigma and alpha; the update with the stop / pause tests; the direction.
// partial holds pressure_partials() doubles.
cudaError_t launch_pcg_psig(const double* q, const double* w, int64_t n, PcgState* st, double* partial,
                            cudaStream_t s);
cudaError_t launch_pcg_pupd(bool jac, bool mixed, double* x, double* r, const double* q, const double* w,
                            const double* dinv, double* z, int64_t n, PcgState* st, double* partial, double gamma2,
                            int gap, cudaStream_t s);
cudaError_t launch_pcg_pdir(double* q, const double* zd, int64_t n, const PcgState* st, cudaStream_t s);
int pressure_partials();
// z = dinv r; *out = sum z
cudaError_t launch_pscale(const double* r, const double* dinv, double* z, int64_t n, double* partial, double* out,
                          cudaStream_t s);
cudaError_t launch_pshift_dot(double* w, const double* p, double c, int64_t n, double* partial, double* out,
                              cudaStream_t s);
cudaError_t launch_pdir(double* y, const double* a, double beta, int64_t n, cudaStream_t s);
cudaError_t launch_pstart(const double* g, double c, double* r, double* p, double* x, int64_t n, double* partial,
                          double* out, cudaStream_t s);
}  // namespace sem
