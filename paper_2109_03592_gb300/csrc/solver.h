// Solver-side entry points used by api.cpp.
#pragma once

#include "sem_internal.h"

namespace sem {

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  double h1 = NAN, h2 = NAN;
  int var = -1, df = -1;
  uint64_t coef_gen = 0;  // the mesh's coefficient generation (the graph holds its array pointers)
  int nodes = 0;          // kernel launches per graph launch
};

struct Workspace {
  int64_t n = 0;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *minv = nullptr, *b = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *w32 = nullptr, *minv32 = nullptr;
  float* p32b = nullptr;  // the FP32 CG's second direction buffer (directions alternate between p32 and p32b)
  double* pb = nullptr;   // the FP64 CG's second direction buffer (with p)
  PcgState* st = nullptr;
  PcgState* sth = nullptr;  // pinned host [2]
  double* part_ax = nullptr;
  double* part_vec = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, eu = nullptr, ev[2] = {nullptr, nullptr};
  double minv_h1 = NAN, minv_h2 = NAN;
  GraphSlot g64, g32;
};

sem_status alloc_ws(sem_mesh* m, Workspace** out);
void free_ws(Workspace* ws);  // a workspace from alloc_ws that is not a mesh's
// FP64 local operator with the mesh's tuned kernel (native or double-float).
// w = A_L u with the native FP64 kernel (exact FP64 arithmetic)
cudaError_t ax64_exact(const sem_mesh* m, const double* u, double* w, double h1, double h2, cudaStream_t s);
// FP32 local operator with the mesh's tuned kernel (fused: the CG prologue and <p, A_L p>;
// pout, when given, receives the new direction z + beta p instead of p).
cudaError_t ax32(const sem_mesh* m, const float* u, float* w, double h1, double h2, bool fused, const float* z,
                 float* p, PcgState* st, double* part, cudaStream_t s, float* pout = nullptr);
cudaError_t ax64(const sem_mesh* m, const double* u, double* w, double h1, double h2, bool fused, const double* z,
                 double* p, PcgState* st, double* part, cudaStream_t s, double* pout = nullptr);
// Write a fresh PcgState (tol, maxit, done) to ws->st / read it back (both synchronise ws->s).
sem_status put_state(Workspace* ws, double tol, int maxit, int done);
sem_status read_state(Workspace* ws, PcgState& out);
// Replay a captured chunk graph until the device state reports done (double-buffered polling).
sem_status run_chunks(Workspace* ws, const GraphSlot& gs, int maxit, PcgState& out);
constexpr int kSolveChunk = 8;  // CG iterations per graph launch

// w = A_L u with the mesh's tuned kernel for `prec` (SEM_FP64 or SEM_FP32).
sem_status apply_local(const sem_mesh* m, const void* u, void* w, double h1, double h2, sem_prec prec,
                       cudaStream_t s);
// Time the kernel variants of the local operator on this mesh and keep the fastest.
sem_status autotune_mesh(sem_mesh* m, cudaStream_t s);
void release_workspace(sem_mesh* m);

}  // namespace sem
