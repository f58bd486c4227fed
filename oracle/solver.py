"""Assembled operator, right-hand side, Jacobi preconditioner and PCG.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2: the Helmholtz problem (Eq. 4) and the pressure Poisson problem
(Eq. 5) are solved "using iterative solvers with proper preconditioners".
The reading taken here (the paper fixes none of these details):

* assembled operator  A x = mask * QQ^T A_L x  (x continuous, zero on
  Dirichlet nodes); right-hand side  b = mask * QQ^T (B f);
* inner product  <a, b> = sum_l a_l b_l / mult_l  over local points, which
  equals the plain dot product over global nodes;
* Jacobi preconditioner  M^{-1} = mask / (QQ^T diag(A_L))  (exact diagonal);
* preconditioned CG (Hestenes-Stiefel), x0 = 0 by default, stopped when
  ||r|| <= tol ||b|| in the norm above, tol = 1e-10, maxit = 20000;
* mixed precision: an FP64 outer iterative refinement r = b - A x around an
  inner PCG run entirely on FP32 copies of G, B, M^{-1} and the fields, whose
  inner products are FP32 products summed in FP64 -- either restarted at
  every refinement step (``pcg_mixed``, classic defect correction) or keeping
  the CG direction across refinements (``pcg_mixed_reliable``: "reliable
  updates", Sleijpen & van der Vorst, Computing 56 (1996); Clark et al.,
  Comput. Phys. Commun. 181 (2010), Sec. 4).
"""

import numpy as np

from . import geometry, gll, numbering
from .operator import ax_local, local_diagonal

CONVERGED, NOT_CONVERGED, BREAKDOWN = 0, 4, 5


def _coefficient(h):
    """A scalar, or one value per local point [E, n, n, n] (Alg. 1 reads
    h1(i,j,k,e); h2 per point likewise)."""
    return float(h) if np.ndim(h) == 0 else np.asarray(h, dtype=np.float64)


class Problem:
    """Everything the solver needs for one mesh and one (h1, h2), each a
    scalar or an array of per-local-point values."""

    def __init__(self, mesh, h1=1.0, h2=0.0):
        self.mesh = mesh
        self.h1, self.h2 = _coefficient(h1), _coefficient(h2)
        self.D = gll.derivative_matrix(mesh.N)
        self.G, self.B, self.detJ = geometry.factors(mesh)
        self.glo, self.Pg = numbering.global_numbering(mesh)
        self.mult = numbering.multiplicity(self.glo, self.Pg).reshape(self.B.shape)
        self.mask = numbering.dirichlet_mask(mesh, self.glo, self.Pg).reshape(self.B.shape)
        self.shape = self.B.shape

    # -- Sec. 2: global (QQ^T) and local (A_L) operations ------------------
    def gs(self, v):
        return numbering.gs(v, self.glo, self.Pg)

    def A(self, x):
        return self.mask * self.gs(ax_local(x, self.G, self.B, self.D, self.h1, self.h2))

    def rhs(self, f):
        return self.mask * self.gs(self.B * f)

    def jacobi_inverse(self):
        d = self.gs(local_diagonal(self.G, self.B, self.D, self.h1, self.h2))
        d = np.where(self.mask > 0, d, 1.0)
        return self.mask / d

    def dot(self, a, b):
        return float(np.sum(a * b / self.mult))

    def dense(self):
        """Dense assembled matrix on the free global nodes (tiny meshes only):
        column g is A applied to the continuous unit vector of node g."""
        glo = self.glo.reshape(self.shape)
        free = np.unique(self.glo[self.mask.reshape(-1) > 0])
        rep = np.full(self.Pg, -1)
        rep[self.glo[::-1]] = np.arange(self.glo.size)[::-1]  # first copy of each node
        A = np.zeros((free.size, free.size))
        for c, g in enumerate(free):
            x = (glo == g).astype(np.float64)
            y = self.A(x).reshape(-1)
            A[:, c] = y[rep[free]]
        return A, free, rep


class Result:
    def __init__(self, x, iters, rel_res, status, history, outer_iters=0):
        self.x, self.iters, self.rel_res = x, iters, rel_res
        self.status, self.history, self.outer_iters = status, history, outer_iters


def pcg(prob, b, x0=None, tol=1e-10, maxit=20000):
    """Jacobi-preconditioned CG on the assembled system A x = b (FP64)."""
    Minv = prob.jacobi_inverse()
    x = np.zeros(prob.shape) if x0 is None else prob.mask * x0
    r = b - prob.A(x)
    bnorm = np.sqrt(prob.dot(b, b))
    if bnorm == 0.0:
        return Result(np.zeros(prob.shape), 0, 0.0, CONVERGED, [])
    rnorm = np.sqrt(prob.dot(r, r))
    hist = [rnorm / bnorm]
    if rnorm <= tol * bnorm:
        return Result(x, 0, rnorm / bnorm, CONVERGED, hist)
    z = Minv * r
    p = z.copy()
    rho = prob.dot(r, z)
    for k in range(1, maxit + 1):
        w = prob.A(p)
        sigma = prob.dot(p, w)
        if not sigma > 0.0:
            return Result(x, k, rnorm / bnorm, BREAKDOWN, hist)
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * w
        rnorm = np.sqrt(prob.dot(r, r))
        hist.append(rnorm / bnorm)
        if rnorm <= tol * bnorm:
            return Result(x, k, rnorm / bnorm, CONVERGED, hist)
        z = Minv * r
        rho_new = prob.dot(r, z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return Result(x, maxit, rnorm / bnorm, NOT_CONVERGED, hist)


class Problem32:
    """FP32 copies of a Problem's operator data (rounded to nearest)."""

    def __init__(self, prob):
        self.prob = prob
        self.G = prob.G.astype(np.float32)
        self.B = prob.B.astype(np.float32)
        self.D = prob.D.astype(np.float32)
        self.mask = prob.mask.astype(np.float32)
        self.Minv = prob.jacobi_inverse().astype(np.float32)
        self.h1 = np.asarray(prob.h1, dtype=np.float32)
        self.h2 = np.asarray(prob.h2, dtype=np.float32)

    def A(self, x):
        w = ax_local(x, self.G, self.B, self.D, self.h1, self.h2).astype(np.float32)
        return self.mask * self.prob.gs(w)

    def dot(self, a, b):
        """FP32 products, summed in FP64."""
        return float(np.sum((a * b).astype(np.float64) / self.prob.mult))


def pcg32(p32, b32, tol, maxit):
    """PCG as in ``pcg`` on FP32 fields (x0 = 0); returns (x32, iters, status)."""
    x = np.zeros(p32.prob.shape, dtype=np.float32)
    r = b32.copy()
    bnorm = np.sqrt(p32.dot(b32, b32))
    if bnorm == 0.0:
        return x, 0, CONVERGED
    z = p32.Minv * r
    p = z.copy()
    rho = p32.dot(r, z)
    for k in range(1, maxit + 1):
        w = p32.A(p)
        sigma = p32.dot(p, w)
        if not sigma > 0.0:
            return x, k, BREAKDOWN
        alpha = np.float32(rho / sigma)
        x = x + alpha * p
        r = r - alpha * w
        if np.sqrt(p32.dot(r, r)) <= tol * bnorm:
            return x, k, CONVERGED
        z = p32.Minv * r
        rho_new = p32.dot(r, z)
        beta = np.float32(rho_new / rho)
        rho = rho_new
        p = z + beta * p
    return x, maxit, NOT_CONVERGED


def pcg_mixed(prob, b, tol=1e-10, inner_tol=1e-5, max_outer=50, maxit=20000):
    """FP64 iterative refinement around the FP32 inner PCG:
    r = b - A64 x;  d = PCG32(r / ||r||);  x += ||r|| d;  until ||r|| <= tol ||b||."""
    p32 = Problem32(prob)
    x = np.zeros(prob.shape)
    bnorm = np.sqrt(prob.dot(b, b))
    if bnorm == 0.0:
        return Result(x, 0, 0.0, CONVERGED, [])
    r = b.copy()
    rnorm = bnorm
    hist, total, outer = [1.0], 0, 0
    while rnorm > tol * bnorm and outer < max_outer:
        d, it, st = pcg32(p32, (r / rnorm).astype(np.float32), inner_tol, maxit)
        total += it
        if st == BREAKDOWN:
            return Result(x, total, rnorm / bnorm, BREAKDOWN, hist, outer)
        x = x + rnorm * d.astype(np.float64)
        r = b - prob.A(x)
        rnorm = np.sqrt(prob.dot(r, r))
        hist.append(rnorm / bnorm)
        outer += 1
    st = CONVERGED if rnorm <= tol * bnorm else NOT_CONVERGED
    return Result(x, total, rnorm / bnorm, st, hist, outer)


def pcg_mixed_reliable(prob, b, tol=1e-10, delta=0.3, maxit=20000, gamma=0.2):
    """Mixed-precision PCG with reliable updates.

    The CG recurrences run in FP32 on the scaled system (b / ||b||): x32 holds
    the solution increment since the last reliable update.  Whenever the FP32
    iterated residual has dropped below delta times its largest value since
    that update (or below gamma * tol: the FP32 residual must undershoot the
    target, otherwise a true residual just above tol triggers a replacement
    after every few steps and stalls), the increment is added to the FP64
    solution, the true residual r = b - A64 x is recomputed in FP64 and
    replaces the FP32 one, and CG continues with its current direction p:
    z = M^{-1} r, beta = <r,z>_new / <r,z>_old, p = z + beta p.  The solve stops
    when the FP64 true residual meets the tolerance."""
    p32 = Problem32(prob)
    x = np.zeros(prob.shape)
    bnorm = np.sqrt(prob.dot(b, b))
    if bnorm == 0.0:
        return Result(x, 0, 0.0, CONVERGED, [])
    s = 1.0 / bnorm
    r = (b * s).astype(np.float32)
    x32 = np.zeros(prob.shape, dtype=np.float32)
    z = p32.Minv * r
    p = np.zeros(prob.shape, dtype=np.float32)
    rho = p32.dot(r, z)
    beta = np.float32(0.0)
    rr_max = p32.dot(r, r)
    hist, updates = [1.0], 0
    for k in range(1, maxit + 1):
        p = z + beta * p
        w = p32.A(p)
        sigma = p32.dot(p, w)
        if not sigma > 0.0:
            return Result(x + x32.astype(np.float64) / s, k, hist[-1], BREAKDOWN, hist, updates)
        alpha = np.float32(rho / sigma)
        x32 = x32 + alpha * p
        r = r - alpha * w
        rr = p32.dot(r, r)
        if rr <= delta * delta * rr_max or rr <= (gamma * tol) ** 2:
            x = x + x32.astype(np.float64) / s
            x32[:] = 0.0
            rt = b - prob.A(x)
            rel = np.sqrt(prob.dot(rt, rt)) / bnorm
            hist.append(rel)
            updates += 1
            if rel <= tol:
                return Result(x, k, rel, CONVERGED, hist, updates)
            r = (rt * s).astype(np.float32)
            rr_max = p32.dot(r, r)
        else:
            rr_max = max(rr_max, rr)
        z = p32.Minv * r
        rho_new = p32.dot(r, z)
        beta = np.float32(rho_new / rho)
        rho = rho_new
    x = x + x32.astype(np.float64) / s
    rt = b - prob.A(x)
    return Result(x, maxit, np.sqrt(prob.dot(rt, rt)) / bnorm, NOT_CONVERGED, hist, updates)
