// Internal declarations of the overlapping Schwarz preconditioner (Sec. 2, Eq. 6).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/sem.h"
#include "device_util.cuh"

namespace sem {

// Local fast-diagonalisation solves z_e = W A~_e^{-1} (W r_e), every element.
template <typename T>
struct FdmParams {
  const T* r;            // [E][n^3] local vector
  T* z;                  // [E][n^3] output (before QQ^T)
  const uint8_t* wm;     // multiplicity | 0x80 Dirichlet
  const T* wtab;         // [128] mult^{-1/2}
  const int32_t* sidx;   // [E][3] rows of the distinct 1D tables (r, s, t)
  const T* S;            // [nd][n][n] eigenvectors (row l, column c)
  const T* lam;          // [nd][n] eigenvalues
  T h1, h2;
  int64_t E;
  const PcgState* st;    // nullable: skipped once st->done
  // coarse restriction fused into the same pass over r (nullable rc: none):
  // rc[8 e + v] = sum over the element's points of phi_v r / mult
  const T* ftab;         // [2][n]: (1 -+ xi_k) / 2
  double* rc;
};
template <typename T>
cudaError_t launch_fdm(int N, const FdmParams<T>& p, cudaStream_t s);

// Coarse space of trilinear vertex functions.  ftab [2][n]: (1 -+ xi_k) / 2
// at the GLL nodes in T; xi: the n GLL nodes (FP64, set-up kernels).
template <typename T>
cudaError_t launch_coarse_restrict(const T* r, const uint8_t* wm, const T* ftab, int n, int64_t E, double rscale,
                                   double* rc, const PcgState* st, cudaStream_t s);
cudaError_t launch_coarse_gather(const double* rc, const int32_t* ptr, const int64_t* slots, int nc, double* g,
                                 const PcgState* st, cudaStream_t s);
cudaError_t launch_dense_symv(const double* A, const double* x, int nc, double* y, const PcgState* st, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_prolong(T* z, const uint8_t* wm, const T* ftab, const int32_t* cidx, const double* y, int n,
                                  int64_t E, double zscale, const PcgState* st, cudaStream_t s);
// z += mask R_0^T y (the coarse correction), then rho_new = <r, z>_W and
// beta = rho_new / rho in the CG state (as launch_pcg_rho), in one pass;
// partial = nullptr: the correction only (st nullable).
template <typename T>
cudaError_t launch_prolong_rho(T* z, const T* r, const uint8_t* wm, const T* ftab, const int32_t* cidx,
                               const double* y, int n, int64_t E, PcgState* st, double* partial, cudaStream_t s);
cudaError_t launch_fill_phi(double* u, const uint8_t* wm, const double* xi, int n, int64_t P, int b, cudaStream_t s);
cudaError_t launch_elem_coarse(const double* w, const uint8_t* wm, const double* xi, int n, int64_t E, int b,
                               double* Ae, cudaStream_t s);
cudaError_t launch_gj_inverse(double* M, int nc, double* f, int* bad, cudaStream_t s);

// Approximate coarse solve x = B g for many unknowns: `cycles` symmetric
// V-cycles (Chebyshev smoothing in D^{-1} A_0 of degree deg, aggregate
// correction with the dense inverse of A_00 = P^T A_0 P, Chebyshev smoothing
// again), each a linear step x += B (g - A_0 x) from x = 0.
constexpr int kChebMaxDeg = 16;
struct CoarseCycle {
  int nc = 0, na = 0, deg = 0, cycles = 1, width = 0;
  const int32_t* col = nullptr;  // A_0 in ELL form, slot-major [width][nc]
  const double* val = nullptr;
  const double* dinv = nullptr;  // 1 / diag(A_0)
  const int32_t* agg = nullptr;  // aggregate of each unknown
  const int32_t* aptr = nullptr; // members of each aggregate (CSR, ascending)
  const int32_t* amem = nullptr;
  const double* A00inv = nullptr;
  double *ga = nullptr, *ya = nullptr;  // [na]
  double* work = nullptr;               // [3 nc]
  double cheb_c0 = 0.0;                 // 1 / theta
  double cheb_a[kChebMaxDeg] = {0}, cheb_b[kChebMaxDeg] = {0};
};
cudaError_t launch_vcycle(const CoarseCycle& c, const double* g, double* x, const PcgState* st, cudaStream_t s);
int vcycle_launches(const CoarseCycle& c);

// Host set-up of the local solves (schwarz_host.cpp): the distinct 1D
// problems (S [nd][n][n], lam [nd][n]) and each element's three rows sidx [E][3].
struct FdmTables {
  std::vector<double> S, lam;
  std::vector<int32_t> sidx;
  int64_t nd = 0;
};
sem_status fdm_tables(int64_t E, int N, const int64_t* glo, const double* xyz, const uint8_t* dirichlet_face,
                      FdmTables& out);

}  // namespace sem
