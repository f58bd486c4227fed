"""Plain CPU FP64 oracle for the SEM Poisson/Helmholtz hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle restates, slowly and directly, what the method of Vincent et al.,
"Strong Scaling of OpenACC enabled Nek5000 on several GPU based HPC systems"
(arXiv 2109.03592) computes on its hot path:

* GLL nodes, weights and the derivative matrix D (Sec. 2, SEM discretisation
  with Lagrange interpolants on Gauss-Lobatto-Legendre points) -- ``gll``.
* Box and O-grid pipe meshes (Sec. 4.2 flow case; synthetic stand-in) --
  ``mesh``.
* Geometric factors g1..g6 and the mass B (used by Alg. 1) -- ``geometry``.
* The matrix-free local operator of Alg. 1 plus the Helmholtz mass term of
  Sec. 2, Eq. 4 -- ``operator``.
* Global numbering, direct stiffness summation QQ^T ("exchange of element
  face values", Sec. 2) and the Dirichlet mask -- ``numbering``.
* Jacobi-preconditioned CG and FP32-inner / FP64-outer iterative
  refinement (Sec. 2: "iterative solvers with proper preconditioners") --
  ``solver``.
* Projection onto previous solutions (Sec. 2, Fischer 1998) -- ``projection``.
* The staggered P_N - P_{N-2} pressure space (GL points), the weak divergence
  and gradient, and the consistent Poisson operator E = D B^{-1} D^T of
  Sec. 2, Eq. 5 -- ``pressure``.
* The overlapping Schwarz preconditioner with a coarse grid of Sec. 2,
  Eq. 6 (fast-diagonalisation local solves) -- ``schwarz``.

Each function cites the passage it follows.  No code here is shared with the
CUDA path; the two meet only through ``sem_inputs`` (seeded random draws and
mesh descriptors, which contain none of the method's arithmetic).
"""

from . import gll, mesh, geometry, operator, numbering, solver, pressure, schwarz  # noqa: F401
