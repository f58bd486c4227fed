"""Projection onto previous solutions for successive right-hand sides.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2 (the paragraph on the velocity and pressure solves) accelerates the
iterative solves by projecting each new solution onto the space spanned by
previous solutions (its reference: Fischer 1998).  The paper gives no more
detail; the reading written out here is the textbook form of that method:

* the space is kept as a basis X = [x_1 .. x_l] that is A-orthonormal in the
  global inner product, x_i^T A x_j = delta_ij, together with A x_i;
* for a new b, the best approximation to A^{-1} b in the A-norm from span(X)
  is xbar = sum_i (x_i^T b) x_i (since x_i^T A A^{-1} b = x_i^T b);
* CG then solves A x = b from the initial guess xbar, to the usual relative
  tolerance ||b - A x|| <= tol ||b||;
* the increment dx = x - xbar is A-orthogonalised against X by classical
  Gram-Schmidt, run twice (in exact arithmetic dx is already A-orthogonal to
  X, because X^T (b - A xbar) = 0; the passes remove what rounding and the
  inexact solve leave), A-normalised and appended;
* when the basis already holds max_vectors vectors, it restarts from the new
  solution alone, x / ||x||_A.
"""

import numpy as np

from . import solver


class Projection:
    """A-orthonormal basis of earlier solutions of A x = b for one operator."""

    def __init__(self, prob, max_vectors):
        if max_vectors < 1:
            raise ValueError("max_vectors must be >= 1")
        self.prob = prob
        self.max_vectors = max_vectors
        self.X = []   # basis vectors (local layout, equal on copies, zero on Dirichlet nodes)
        self.AX = []  # the assembled operator applied to each

    def guess(self, b):
        """xbar = sum_i (x_i^T b) x_i and the coefficients x_i^T b."""
        xbar = np.zeros(self.prob.shape)
        coef = [self.prob.dot(x, b) for x in self.X]
        for c, x in zip(coef, self.X):
            xbar = xbar + c * x
        return xbar, coef

    def _append(self, v):
        """A-orthogonalise v against the basis (two classical Gram-Schmidt
        passes), A-normalise it and append it; returns False if nothing of v
        is left."""
        P = self.prob
        for _ in range(2):
            beta = [P.dot(ax, v) for ax in self.AX]
            for c, x in zip(beta, self.X):
                v = v - c * x
        Av = P.A(v)
        nrm2 = P.dot(v, Av)
        if not nrm2 > 0.0:
            return False
        nrm = np.sqrt(nrm2)
        self.X.append(v / nrm)
        self.AX.append(Av / nrm)
        return True

    def solve(self, b, tol=1e-10, maxit=20000):
        """Solve A x = b from the projected initial guess and add the new
        direction to the basis.  Returns the oracle's PCG result (iters counts
        the CG iterations after the projection)."""
        xbar, _ = self.guess(b)
        res = solver.pcg(self.prob, b, x0=xbar, tol=tol, maxit=maxit)
        if res.status != solver.CONVERGED:
            return res
        if len(self.X) >= self.max_vectors:
            self.X, self.AX = [], []
            self._append(res.x.copy())
        else:
            self._append(res.x - xbar)
        return res
