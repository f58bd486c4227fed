// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sem.h"
#include "kernels.h"

namespace sem {

// A named range on the NVTX timeline of the Nsight tools for the lifetime of
// the object (each C-ABI call opens one); without a tool attached the calls
// return at once.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define SEM_TRACE(name) ::sem::TraceRange sem_trace_range_(name)

constexpr int kMaxN = 11;  // highest polynomial order compiled

// Thread-local error text behind sem_last_error().
void set_error(const std::string& msg);
sem_status cuda_fail(cudaError_t err, const char* what);

#define SEM_CUDA(call)                                              \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) return ::sem::cuda_fail(_e, #call);      \
  } while (0)

// ---- host-side mesh construction (topo.cpp) --------------------------------

// GLL nodes, weights and derivative matrix D[i*n + l] = l_l'(xi_i), n = N+1.
void gll(int N, std::vector<double>& xi, std::vector<double>& w, std::vector<double>& D);

// Corner vertex ids [E][8] of the built-in generators.
sem_status generator_vertices(const sem_mesh_desc& d, std::vector<int64_t>& vert, int64_t& E);
// Per-element Dirichlet face flags [E][6] of the built-in generators.
void generator_dirichlet(const sem_mesh_desc& d, int64_t E, std::vector<uint8_t>& dface);

struct Topology {
  int64_t E = 0;
  int N = 0;
  int64_t n_local = 0;
  int64_t n_global = 0;
  std::vector<int64_t> glo;  // [n_local] first-touch global ids
};
sem_status build_numbering(int64_t E, int N, const int64_t* vert, Topology& t);

// Gather-scatter plan.  Nodes with m > 1 copies, in ascending global id,
// are grouped by m: for m = 2..8 (classes 0..6) each node is a fixed tuple
// of its m local indices in ascending order; nodes with m > 8 form a CSR
// class (7); Dirichlet nodes with a single copy form class 8 (one index
// each).  Bit 31 of a node's first index flags a Dirichlet node.  Every
// class starts at a multiple of 4 entries of `idx` (16-byte aligned).
constexpr int kGsClasses = 9;
constexpr int kGsUnitNodes = 256;        // nodes per work unit (one per thread of a CTA)
constexpr int64_t kGsWindow = 1 << 21;   // global ids per ordering window
struct GsPlan {
  std::vector<int32_t> idx;
  std::vector<int32_t> gptr;             // CSR offsets (relative to the class start) of class 7
  int64_t off[kGsClasses] = {0};         // class start in idx
  int64_t cnt[kGsClasses] = {0};         // nodes per class
  int64_t n_nodes = 0, n_points = 0;     // shared-or-Dirichlet nodes and their local points
  // Work units of the gather-scatter kernel, in processing order: up to
  // kGsUnitNodes consecutive nodes of one class, {class, first node within
  // the class, node count, 0}.  Units are ordered window by window over the
  // global ids (kGsWindow ids each) and class by class inside a window, so the
  // face, edge and vertex nodes that share the same rows of the same
  // elements are processed close together in time (their sectors are still
  // in L2), instead of in one pass per class over the whole vector.
  std::vector<int32_t> units;
  std::vector<uint8_t> wm;               // per local point: multiplicity | 0x80 if Dirichlet
};
sem_status build_gs_plan(const Topology& t, const uint8_t* dirichlet_face, GsPlan& plan);

// ---- device-side mesh ------------------------------------------------------

struct Workspace;

}  // namespace sem

struct sem_mesh {
  int device = 0;
  int N = 0, n = 0;
  int64_t E = 0, n_local = 0, n_global = 0;
  int64_t n_seg = 0, n_seg_points = 0;
  size_t dev_bytes = 0;

  std::vector<int64_t> glo;    // host copy of the global ids
  std::vector<uint8_t> dface;  // host copy of the Dirichlet face flags [E][6]

  // device arrays (library-owned)
  double* xyz = nullptr;     // [E][3][n3]
  double* G64 = nullptr;     // [E][6][n3]
  double* B64 = nullptr;     // [E][n3]
  float* G32 = nullptr;      // [E][6][n3] round-to-nearest of G64 (the "hi" part)
  float* G32lo = nullptr;    // [E][6][n3] float(G64 - G32): G64 ~ G32 + G32lo to 2^-48
  float* B32 = nullptr;      // [E][n3] round-to-nearest of B64
  float* B32lo = nullptr;    // [E][n3] float(B64 - B32)
  double* dK = nullptr;      // [n_local] QQ^T diag of the stiffness (h1 = 1, h2 = 0)
  double* dB = nullptr;      // [n_local] QQ^T B
  uint8_t* wm = nullptr;     // [n_local] multiplicity | 0x80 Dirichlet
  int32_t* gs_idx = nullptr;   // GsPlan::idx
  int32_t* gs_ptr = nullptr;   // GsPlan::gptr
  int32_t* gs_units = nullptr; // GsPlan::units
  int64_t gs_nunits = 0;
  int64_t gs_off[9] = {0}, gs_cnt[9] = {0};
  int* dev_err = nullptr;    // device error word of the bulk-copy kernels (0 = ok)
  double* D64 = nullptr;     // [n*n] D (row i: d/dr at xi_i)
  float* D32 = nullptr;
  float* D32lo = nullptr;
  // even-odd coefficients of D and D^T (even n only), [2][h][h] with h = n/2:
  // (Ep, Em) = (D[i][l] +- D[i][n-1-l]) / 2 for D, then the same for D^T;
  // eo64 in FP64 (pairs), eodf split into (Ep.hi, Ep.lo, Em.hi, Em.lo)
  double* eo64 = nullptr;
  float* eodf = nullptr;

  // per-point coefficients (sem_mesh_set_coefficients): cG = h1[q] G and
  // cB = h2[q] B in the operator's precisions, with their assembled
  // diagonals; null while the coefficient is constant.  coef_gen counts the
  // changes, so cached data derived from the operator can tell it is stale.
  double* cG64 = nullptr;
  float* cG32 = nullptr;
  float* cG32lo = nullptr;
  double* cdK = nullptr;
  double* cB64 = nullptr;
  float* cB32 = nullptr;
  float* cB32lo = nullptr;
  double* cdB = nullptr;
  uint64_t coef_gen = 0;

  // the operator's arrays: the plain geometry, or its per-point copies
  const double* opG64() const { return cG64 ? cG64 : G64; }
  const float* opG32() const { return cG64 ? cG32 : G32; }
  const float* opG32lo() const { return cG64 ? cG32lo : G32lo; }
  const double* opdK() const { return cG64 ? cdK : dK; }
  const double* opB64() const { return cB64 ? cB64 : B64; }
  const float* opB32() const { return cB64 ? cB32 : B32; }
  const float* opB32lo() const { return cB64 ? cB32lo : B32lo; }
  const double* opdB() const { return cB64 ? cdB : dB; }

  // local-operator kernel choice, set by the autotuner at creation:
  // variant index per precision (0 FP64 native, 1 FP32, 2 FP64 double-float)
  // and whether FP64 requests run the double-float kernel.
  int ax_var[3] = {0, 0, 0};
  int ax_var_dff = 0;           // double-float variant of the fused form (the FP64 CG's operator)
  int fp64_df = 0;
  float ax_ms[3][4] = {{0}};

  // P_N - P_{N-2} pressure operators (pressure_api.cpp), built on first use
  // under p_mutex: GL-point factors F [E][9][m^3] (rho^3 adj(J)_{ba}, index
  // 3 b + a) and the GLL basis values / derivatives at the GL points [m][n]
  mutable std::mutex p_mutex;
  mutable double* pdinv = nullptr;  // [E m^3] 1 / diag(E), the pressure CG's Jacobi preconditioner
  mutable double* Fgl = nullptr;
  mutable double* Igl = nullptr;
  mutable double* DIgl = nullptr;
  // their FP32 copies and the reciprocal assembled mass [n_local], for the
  // FP32 operator of the mixed-precision pressure solve (built on first use)
  mutable float* Fgl32 = nullptr;
  mutable float* Igl32 = nullptr;
  mutable float* DIgl32 = nullptr;
  mutable float* invB32 = nullptr;

  std::mutex ws_mutex;
  sem::Workspace* ws = nullptr;  // cached solver workspace
  // workspaces of further right-hand sides on this mesh in one batch, kept
  // for the next batch (guarded by ws_mutex; freed with the mesh)
  std::vector<sem::Workspace*> spare_ws;
};

namespace sem {
inline GsDev gs_dev(const sem_mesh* m) {
  GsDev g;
  g.idx = m->gs_idx;
  g.gptr = m->gs_ptr;
  g.units = reinterpret_cast<const int4*>(m->gs_units);
  g.nunits = m->gs_nunits;
  for (int c = 0; c < 9; ++c) {
    g.off[c] = m->gs_off[c];
    g.cnt[c] = m->gs_cnt[c];
  }
  return g;
}
}  // namespace sem
