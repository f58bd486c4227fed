"""GB300 (sm_103a) SEM Poisson/Helmholtz hot path: matrix-free Ax (Alg. 1),
gather-scatter QQ^T and Jacobi PCG behind the C ABI of include/sem.h."""

from .sem import (FP32, FP64, MIXED, Mesh, Projection, Schwarz, SemError, Server, gs_halo, lib, mesh_vertices,  # noqa: F401
                  topology_numbering, kernel_launches, solve_batch, pressure_basis)
from .sem import PRECOND_DEFAULT, PRECOND_NONE, PRECOND_JACOBI  # noqa: F401
from .sem import (SEM_OK, SEM_ERR_INVALID, SEM_ERR_OOM, SEM_ERR_CUDA, SEM_ERR_NOT_CONVERGED,  # noqa: F401
                  SEM_ERR_BREAKDOWN, SEM_ERR_BUSY, SEM_ERR_DEVICE_TIMEOUT, SEM_ERR_BAD_MESH, SEM_ERR_TIMEOUT,
                  SEM_ERR_NOT_FOUND, SEM_ERR_CANCELLED)
