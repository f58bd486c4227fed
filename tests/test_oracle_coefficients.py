"""Pins for per-point coefficients h1(i,j,k,e), h2(i,j,k,e) in the oracle's
local operator (Alg. 1 reads h1 per local point; the h2 mass term of Sec. 2,
Eq. 4, per point likewise).

On affine (box) elements, GLL quadrature with N+1 points per direction
integrates polynomials of degree <= 2N-1 per direction exactly, so for
polynomials u, v of degree <= N and polynomial coefficients h1, h2

    sum_e v_e . (A_L u)_e = integral over the box of (h1 grad u . grad v + h2 u v)

up to rounding.  The integrals are taken in closed form from the monomials.
h1 and h2 treat x, y and z differently, so a coefficient read at a transposed
or shifted point fails the pin.
"""

import numpy as np
import pytest

from oracle import geometry, gll, mesh, operator, solver
from sem_inputs import coefficients, forcing, vectors


class Poly:
    """Polynomial in x, y, z as {(a, b, c): coefficient}."""

    def __init__(self, terms):
        self.t = {k: float(v) for k, v in terms.items() if v != 0}

    def __add__(self, o):
        t = dict(self.t)
        for k, v in o.t.items():
            t[k] = t.get(k, 0.0) + v
        return Poly(t)

    def __mul__(self, o):
        t = {}
        for (a, b, c), v in self.t.items():
            for (p, q, r), w in o.t.items():
                k = (a + p, b + q, c + r)
                t[k] = t.get(k, 0.0) + v * w
        return Poly(t)

    def d(self, axis):
        t = {}
        for k, v in self.t.items():
            if k[axis]:
                kk = list(k)
                kk[axis] -= 1
                t[tuple(kk)] = t.get(tuple(kk), 0.0) + v * k[axis]
        return Poly(t)

    def degree(self, axis):
        return max((k[axis] for k in self.t), default=0)

    def integral(self, hi):
        """Over [0, hi[0]] x [0, hi[1]] x [0, hi[2]]."""
        return sum(v * np.prod([hi[a] ** (k[a] + 1) / (k[a] + 1) for a in range(3)]) for k, v in self.t.items())

    def at(self, xyz):
        """Values at nodal coordinates xyz [E, 3, n, n, n] -> [E, n, n, n]."""
        out = np.zeros(xyz.shape[:1] + xyz.shape[2:])
        for (a, b, c), v in self.t.items():
            out += v * xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c
        return out


U = Poly({(2, 1, 0): 1.0, (0, 0, 1): 1.0, (0, 0, 0): -0.5})                  # x^2 y + z - 1/2
V = Poly({(1, 1, 1): 1.0, (0, 2, 0): 1.0, (1, 0, 0): -0.3})                  # x y z + y^2 - 0.3 x
H1 = Poly({(0, 0, 0): 1.0, (1, 0, 0): 0.5, (0, 1, 1): 0.25, (0, 0, 1): 0.1})  # 1 + x/2 + y z/4 + z/10
H2 = Poly({(0, 0, 0): 2.0, (1, 0, 1): 1.0, (0, 1, 0): 0.3})                  # 2 + x z + 0.3 y
L = (1.5, 2.0, 0.75)


def _energy(N, h1, h2):
    m = mesh.box(2, 3, 2, N, *L)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(N)
    u, v = U.at(m.xyz), V.at(m.xyz)
    return float(np.sum(v * operator.ax_local(u, G, B, D, h1(m.xyz), h2(m.xyz)))), m


def _exact(h1, h2):
    grad = sum(((U.d(a) * V.d(a)) for a in range(3)), Poly({}))
    return (h1 * grad).integral(L) + (h2 * U * V).integral(L)


@pytest.mark.parametrize("N", [3, 4])
def test_per_point_coefficients_integrate_exactly(N):
    grad = sum(((U.d(a) * V.d(a)) for a in range(3)), Poly({}))
    for a in range(3):  # GLL exactness and u, v in the discrete space
        assert (H1 * grad).degree(a) <= 2 * N - 1 and (H2 * U * V).degree(a) <= 2 * N - 1
        assert U.degree(a) <= N and V.degree(a) <= N
    got, _ = _energy(N, H1.at, H2.at)
    want = _exact(H1, H2)
    assert abs(got - want) <= 1e-12 * abs(want)
    # stiffness and mass separately
    got_k, _ = _energy(N, H1.at, lambda xyz: 0.0)
    assert abs(got_k - (H1 * grad).integral(L)) <= 1e-12 * abs(want)


def test_pin_rejects_coefficients_at_transposed_points():
    N = 3
    transposed = lambda xyz: np.ascontiguousarray(H1.at(xyz).transpose(0, 3, 2, 1))  # noqa: E731
    got, _ = _energy(N, transposed, H2.at)
    want = _exact(H1, H2)
    assert abs(got - want) > 1e-6 * abs(want)
    shifted = lambda xyz: np.roll(H2.at(xyz), 1, axis=3)  # noqa: E731
    got, _ = _energy(N, H1.at, shifted)
    assert abs(got - want) > 1e-6 * abs(want)


def test_constant_arrays_equal_scalars():
    m = mesh.pipe(2, 1, 2, 4, L=2.0)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(4)
    u = vectors.local_field(3, m.E, 5)
    c1, c2 = np.full(u.shape, 0.7), np.full(u.shape, 3.0)
    w_arr = operator.ax_local(u, G, B, D, c1, c2)
    w_sc = operator.ax_local(u, G, B, D, 0.7, 3.0)
    assert np.abs(w_arr - w_sc).max() <= 1e-14 * np.abs(w_sc).max()
    d_arr = operator.local_diagonal(G, B, D, c1, c2)
    d_sc = operator.local_diagonal(G, B, D, 0.7, 3.0)
    assert np.abs(d_arr - d_sc).max() <= 1e-14 * np.abs(d_sc).max()


def test_diagonal_with_per_point_coefficients_matches_unit_vectors():
    N = 4
    n = N + 1
    m = mesh.pipe(2, 1, 1, N, L=2.0)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(N)
    h1 = coefficients.viscosity(5, m.xyz)
    h2 = coefficients.mass_coefficient(6, m.xyz)
    diag = operator.local_diagonal(G, B, D, h1, h2)
    e = 1
    for q in range(n ** 3):
        u = np.zeros((m.E, n, n, n))
        u[e].reshape(-1)[q] = 1.0
        w = operator.ax_local(u, G, B, D, h1, h2)
        assert abs(w[e].reshape(-1)[q] - diag[e].reshape(-1)[q]) <= 1e-13 * abs(diag[e].reshape(-1)[q])


def test_symmetry_positivity_and_constants_on_curved_pipe():
    N = 5
    m = mesh.pipe(2, 2, 2, N, L=2.0)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(N)
    h1 = coefficients.viscosity(7, m.xyz)
    assert h1.min() > 0 and np.ptp(h1) > 0.5
    u = vectors.local_field(1, m.E, N + 1)
    v = vectors.local_field(2, m.E, N + 1)
    for h2 in (0.0, coefficients.mass_coefficient(8, m.xyz)):
        a = float(np.sum(v * operator.ax_local(u, G, B, D, h1, h2)))
        b = float(np.sum(u * operator.ax_local(v, G, B, D, h1, h2)))
        assert abs(a - b) <= 1e-12 * abs(a)
        assert float(np.sum(u * operator.ax_local(u, G, B, D, h1, h2))) > 0
    ones = np.ones_like(u)
    w = operator.ax_local(ones, G, B, D, h1, 0.0)
    assert np.abs(w).max() < 1e-12 * np.abs(G).max() * h1.max() * (N + 1) ** 2


def test_dense_spd_pcg_with_per_point_coefficients():
    m = mesh.pipe(2, 1, 2, 3, L=2.0)
    h1 = coefficients.viscosity(9, m.xyz)
    h2 = coefficients.mass_coefficient(10, m.xyz)
    P = solver.Problem(m, h1, h2)
    A, free, rep = P.dense()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    np.linalg.cholesky(A)  # raises unless SPD
    Minv = P.jacobi_inverse().reshape(-1)
    np.testing.assert_allclose(1.0 / Minv[rep[free]], np.diag(A), rtol=1e-13)
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(7, L=2.0)))
    res = solver.pcg(P, b)
    assert res.status == solver.CONVERGED and res.rel_res <= 1e-10
    xd = np.linalg.solve(A, b.reshape(-1)[rep[free]])
    assert np.linalg.norm(res.x.reshape(-1)[rep[free]] - xd) <= 1e-9 * np.linalg.norm(xd)
    # the mixed-precision oracle runs on per-point coefficients too
    mix = solver.pcg_mixed_reliable(P, b)
    assert mix.status == solver.CONVERGED and mix.rel_res <= 1e-10
