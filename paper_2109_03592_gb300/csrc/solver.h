// Solver-side entry points used by api.cpp.
#pragma once

#include "sem_internal.h"

namespace sem {

// w = A_L u with the mesh's tuned kernel for `prec` (SEM_FP64 or SEM_FP32).
sem_status apply_local(const sem_mesh* m, const void* u, void* w, double h1, double h2, sem_prec prec,
                       cudaStream_t s);
// Time the kernel variants of the local operator on this mesh and keep the fastest.
sem_status autotune_mesh(sem_mesh* m, cudaStream_t s);
void release_workspace(sem_mesh* m);

}  // namespace sem
