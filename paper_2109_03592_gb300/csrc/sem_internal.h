// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sem.h"

namespace sem {

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

struct GsPlan {
  // Segments are the global nodes with more than one copy or on a Dirichlet
  // face, in ascending global id.  seg_ptr[s]..seg_ptr[s+1] index seg_idx,
  // which lists the segment's local points in ascending local index.
  std::vector<int32_t> seg_ptr;
  std::vector<int32_t> seg_idx;
  std::vector<uint8_t> seg_dir;  // 1 if the node is Dirichlet
  std::vector<uint8_t> wm;       // per local point: multiplicity | 0x80 if Dirichlet
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

  std::vector<int64_t> glo;  // host copy of the global ids

  // device arrays (library-owned)
  double* xyz = nullptr;     // [E][3][n3]
  double* G64 = nullptr;     // [E][6][n3]
  double* B64 = nullptr;     // [E][n3]
  float* G32 = nullptr;      // [E][6][n3] round-to-nearest of G64 (the "hi" part)
  float* G32lo = nullptr;    // [E][6][n3] float(G64 - G32): G64 ~ G32 + G32lo to 2^-48
  float* B32 = nullptr;      // [E][n3]
  double* dK = nullptr;      // [n_local] QQ^T diag of the stiffness (h1 = 1, h2 = 0)
  double* dB = nullptr;      // [n_local] QQ^T B
  uint8_t* wm = nullptr;     // [n_local] multiplicity | 0x80 Dirichlet
  int32_t* seg_ptr = nullptr;
  int32_t* seg_idx = nullptr;
  uint8_t* seg_dir = nullptr;
  double* D64 = nullptr;     // [n*n] D (row i: d/dr at xi_i)
  float* D32 = nullptr;
  float* D32lo = nullptr;

  // local-operator kernel choice, set by the autotuner at creation:
  // variant index per precision (0 FP64 native, 1 FP32, 2 FP64 double-float)
  // and whether FP64 requests run the double-float kernel.
  int ax_var[3] = {0, 0, 0};
  int fp64_df = 0;
  float ax_ms[3][2] = {{0}};

  std::mutex ws_mutex;
  sem::Workspace* ws = nullptr;  // cached solver workspace
};
