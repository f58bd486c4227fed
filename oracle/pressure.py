"""The consistent pressure operator of the staggered P_N - P_{N-2} formulation.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2 discretises velocity with Lagrange interpolants of order N on the GLL
points and pressure with interpolants of order N-2 on the Gauss-Legendre (GL)
points, and solves the consistent Poisson equation for the pressure update
(Sec. 2, Eq. 5).  The paper does not write the discrete operators out; the
reading taken here is the textbook staggered spectral element method
(Maday & Patera 1989; Deville, Fischer & Mund 2002, Sec. 6.3):

* GL points zeta_0 < ... < zeta_{m-1}, m = N - 1: the roots of P_m, with
  weights rho_i = 2 / ((1 - zeta_i^2) P_m'(zeta_i)^2);
* I[i, l]  = l_l(zeta_i)  (GLL Lagrange basis evaluated at the GL points),
  Dg[i, l] = l_l'(zeta_i) (its derivative there);
* at every GL point q of an element, with J_ab = d x_a / d r_b of the
  isoparametric map (the GLL interpolant of the coordinates, differentiated
  and evaluated at q), the nine factors
      F[b, a](q) = rho_i rho_j rho_k det(J) (J^{-1})_{ba}
                 = rho_i rho_j rho_k adj(J)_{ba};
* weak divergence, per element:
      (D u)_q = sum_a sum_b F[b, a](q) (d u_a / d r_b)(zeta_q),
  the GL quadrature of  int psi_q div(u) dx  (psi_q the GL Lagrange basis);
* its transpose D^T (the weak gradient acting on a pressure);
* the consistent Poisson operator on pressures,
      E p = sum_a D_a  M^{-1}  D_a^T p,
  where M^{-1} acts on an element-local velocity component v as
  mask * QQ^T(v) / QQ^T(B): direct stiffness summation, the inverse of the
  assembled (diagonal) GLL mass and the velocity Dirichlet mask.  Pressure is
  discontinuous across elements, so E needs no assembly of its own.

Array conventions: a pressure field is [E, m, m, m] indexed [e, k, j, i]; a
velocity is [3, E, n, n, n] (component-major, each component a local vector).
"""

import numpy as np

from . import gll


def gl_nodes_weights(m):
    """Gauss-Legendre nodes and weights with m points (numpy's leggauss: the
    roots of P_m and rho_i = 2 / ((1 - x_i^2) P_m'(x_i)^2))."""
    if m < 1:
        raise ValueError("GL needs m >= 1")
    return np.polynomial.legendre.leggauss(m)


def lagrange_derivative(x_nodes, l, t):
    """d/dt of the l-th Lagrange cardinal polynomial on x_nodes, at t, by the
    product rule: sum_{q != l} 1/(x_l - x_q) prod_{r != l, q} (t - x_r)/(x_l - x_r).
    Valid at every t, nodes included (GL and GLL points may coincide)."""
    t = np.asarray(t, dtype=np.float64)
    s = np.zeros_like(t)
    for q, xq in enumerate(x_nodes):
        if q == l:
            continue
        term = np.full_like(t, 1.0 / (x_nodes[l] - xq))
        for r, xr in enumerate(x_nodes):
            if r != l and r != q:
                term = term * (t - xr) / (x_nodes[l] - xr)
        s = s + term
    return s


def interpolation_matrices(N):
    """(I [m, n], Dg [m, n], rho [m]): GLL basis values and derivatives at the
    GL points, and the GL weights (m = N - 1, n = N + 1)."""
    if N < 2:
        raise ValueError("the P_N - P_{N-2} pair needs N >= 2")
    xi, _ = gll.nodes_weights(N)
    zeta, rho = gl_nodes_weights(N - 1)
    n = N + 1
    I = np.array([gll.lagrange_eval(xi, l, zeta) for l in range(n)]).T
    Dg = np.array([lagrange_derivative(xi, l, zeta) for l in range(n)]).T
    return I, Dg, rho


def _contract(Mk, Mj, Mi, f):
    """(Mk (x) Mj (x) Mi) applied to f[..., k, j, i]: out[.., K, J, I] =
    sum_{k,j,i} Mk[K, k] Mj[J, j] Mi[I, i] f[.., k, j, i]."""
    return np.einsum("Kk,Jj,Ii,...kji->...KJI", Mk, Mj, Mi, f)


def reference_gradient_gl(N, f):
    """(df/dr, df/ds, df/dt) of element-local GLL fields f[..., n, n, n],
    evaluated at the GL points: [3, ..., m, m, m]."""
    I, Dg, _ = interpolation_matrices(N)
    return np.stack([_contract(I, I, Dg, f), _contract(I, Dg, I, f), _contract(Dg, I, I, f)])


def div_factors(mesh):
    """F[E, 3 (b), 3 (a), m, m, m] = rho_i rho_j rho_k adj(J)_{ba} at the GL
    points, and det(J) there.  Raises ValueError for det(J) <= 0."""
    N = mesh.N
    _, _, rho = interpolation_matrices(N)
    J = np.empty((mesh.E, N - 1, N - 1, N - 1, 3, 3))
    for a in range(3):
        x = mesh.xyz[:, a] - mesh.xyz[:, a, :1, :1, :1]  # D annihilates constants
        g = reference_gradient_gl(N, x)
        for b in range(3):
            J[..., a, b] = g[b]
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("mesh has an element with det(J) <= 0 at a GL point")
    adj = det[..., None, None] * np.linalg.inv(J)  # adj[..., b, a] = det (J^-1)_{ba}
    rho3 = rho[:, None, None] * rho[None, :, None] * rho[None, None, :]
    F = np.einsum("ekjiba,kji->ebakji", adj, rho3)
    return F, det


def div_local(N, F, u):
    """Weak divergence per element: (D u)_q = sum_{a,b} F[b, a](q) (d u_a/d r_b)(q).
    u [3, E, n, n, n] -> [E, m, m, m]."""
    out = 0.0
    for a in range(3):
        g = reference_gradient_gl(N, u[a])
        for b in range(3):
            out = out + F[:, b, a] * g[b]
    return out


def grad_local(N, F, p):
    """The transpose of div_local: u_a = sum_b C_b^T (F[b, a] p), with C_b the
    GL-point derivative along b (interpolation along the other two).
    p [E, m, m, m] -> [3, E, n, n, n]."""
    I, Dg, _ = interpolation_matrices(N)
    mats = [(I.T, I.T, Dg.T), (I.T, Dg.T, I.T), (Dg.T, I.T, I.T)]  # (Mk, Mj, Mi)^T per b
    u = np.zeros((3, p.shape[0]) + (N + 1,) * 3)
    for a in range(3):
        for b in range(3):
            Mk, Mj, Mi = mats[b]
            u[a] += _contract(Mk, Mj, Mi, F[:, b, a] * p)
    return u


class Pressure:
    """The consistent Poisson operator E = D B^{-1} D^T of one mesh, built on
    an ``oracle.solver.Problem`` (its numbering, mask and mass)."""

    def __init__(self, prob):
        self.prob = prob
        self.N = prob.mesh.N
        self.F, self.det = div_factors(prob.mesh)
        self.Bg = prob.gs(prob.B)  # QQ^T B: the assembled GLL mass at every copy
        self.shape = (prob.mesh.E,) + (self.N - 1,) * 3

    def minv(self, v):
        """M^{-1} on one element-local velocity component."""
        return self.prob.mask * self.prob.gs(v) / self.Bg

    def grad(self, p):
        return grad_local(self.N, self.F, p)

    def div(self, u):
        return div_local(self.N, self.F, u)

    def E(self, p):
        g = self.grad(p)
        return self.div(np.stack([self.minv(g[a]) for a in range(3)]))

    def diagonal(self):
        """diag(E), element by element.  Unit pressure q of element e gives
        D_a^T e_q = the row D_a[q, :] on e's GLL points and zero elsewhere;
        QQ^T leaves it unchanged at e's copies (no element holds two copies
        of one node on these meshes), so
            E_qq = sum_a sum_l D_a[q, l]^2 mask_l / (QQ^T B)_l,
        with the rows D_a[q, l] = sum_b F[b, a](q) C_b[q, l] written out
        (C_b: the GL-point derivative along b, interpolation along the other
        two directions).  Pinned against np.diag(dense()) in the tests."""
        N = self.N
        I, Dg, _ = interpolation_matrices(N)
        C = [np.einsum("Kk,Jj,Ii->KJIkji", I, I, Dg),
             np.einsum("Kk,Jj,Ii->KJIkji", I, Dg, I),
             np.einsum("Kk,Jj,Ii->KJIkji", Dg, I, I)]
        wgt = self.prob.mask / self.Bg  # [E, n, n, n]
        d = np.zeros(self.shape)
        for e in range(self.prob.mesh.E):
            for a in range(3):
                row = sum(self.F[e, b, a][:, :, :, None, None, None] * C[b] for b in range(3))
                d[e] += np.einsum("KJIkji,kji->KJI", row * row, wgt[e])
        return d

    def dense(self):
        """Dense E (tiny meshes only), column c = E applied to unit pressure c."""
        P = int(np.prod(self.shape))
        A = np.zeros((P, P))
        for c in range(P):
            p = np.zeros(P)
            p[c] = 1.0
            A[:, c] = self.E(p.reshape(self.shape)).reshape(-1)
        return A


def cg(P, g, tol=1e-10, maxit=20000, max_restarts=5, dinv=None):
    """CG for the pressure equation E p = g (Sec. 2, Eq. 5) on the mean-free
    subspace.  With Dirichlet velocity on the whole boundary the constants
    are the null space of E (exactly so on affine meshes; on curved elements
    GL quadrature leaves them a near-null mode), and the pressure is defined
    up to a constant.  The reading taken here solves
        Pm E Pm p = Pm g,   Pm = I - 1 1^T / n_p   (mean over the GL values),
    plain (unpreconditioned) CG from p = 0 in the Euclidean inner product.
    When the recurrence residual reaches tol ||Pm g||, the true residual
    Pm (g - E p) is formed; the solve stops if it meets the tolerance too,
    and otherwise CG restarts from p with that residual (at most
    ``max_restarts`` times; the paper fixes no stopping rule, and this one
    makes the returned residual the true one).  Returns (p, iterations,
    ||Pm (g - E p)|| / ||Pm g|| -- the recurrence value if not converged --,
    status) with status as in ``solver``.

    dinv (the reciprocal of ``Pressure.diagonal()``): Jacobi-preconditioned
    CG, z = Pm (dinv r) -- scaled, then projected back to the mean-free
    space, so that Pm D^{-1} Pm stays symmetric and positive definite there
    -- with rho = <r, z>; the stopping rule stays on ||r||."""
    from .solver import BREAKDOWN, CONVERGED, NOT_CONVERGED
    gm = g - g.mean()
    gnorm = np.sqrt(np.sum(gm * gm))
    x = np.zeros(P.shape)
    if gnorm == 0.0:
        return x, 0, 0.0, CONVERGED
    def precondition(r):
        if dinv is None:
            return r
        z = dinv * r
        return z - z.mean()

    r = gm.copy()
    z = precondition(r)
    p = z.copy()
    rho = np.sum(r * z)
    restarts = 0
    for k in range(1, maxit + 1):
        w = P.E(p)
        w = w - w.mean()
        sigma = np.sum(p * w)
        if not sigma > 0.0:
            return x, k, np.sqrt(rho) / gnorm, BREAKDOWN
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * w
        rr = np.sum(r * r)
        if np.sqrt(rr) <= tol * gnorm:
            w = P.E(x)
            r = gm - (w - w.mean())
            rr = np.sum(r * r)
            if np.sqrt(rr) <= tol * gnorm:
                return x, k, np.sqrt(rr) / gnorm, CONVERGED
            if restarts == max_restarts:
                return x, k, np.sqrt(rr) / gnorm, NOT_CONVERGED
            restarts += 1
            z = precondition(r)
            p = z.copy()
            rho = np.sum(r * z)
            continue
        z = precondition(r)
        rho_new = np.sum(r * z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, maxit, np.sqrt(rr) / gnorm, NOT_CONVERGED
