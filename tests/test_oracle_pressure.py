"""Pins for the oracle's P_N - P_{N-2} pressure operators (Sec. 2: GL pressure
points; Sec. 2, Eq. 5: the consistent Poisson operator E = D B^{-1} D^T)."""

import numpy as np
import pytest

from oracle import gll, mesh, pressure, solver
from sem_inputs import vectors


@pytest.mark.parametrize("m,nodes,weights", [
    (1, [0.0], [2.0]),
    (2, [-1 / np.sqrt(3), 1 / np.sqrt(3)], [1.0, 1.0]),
    (3, [-np.sqrt(0.6), 0.0, np.sqrt(0.6)], [5 / 9, 8 / 9, 5 / 9]),
])
def test_gl_closed_forms(m, nodes, weights):
    z, r = pressure.gl_nodes_weights(m)
    np.testing.assert_allclose(z, nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(r, weights, rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", [1, 4, 10])
def test_gl_quadrature_exact_to_degree_2m_minus_1(m):
    z, r = pressure.gl_nodes_weights(m)
    for d in range(2 * m):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(r * z ** d) - exact) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 6, 11])
def test_interpolation_and_derivative_at_gl_points(N):
    xi, _ = gll.nodes_weights(N)
    zeta, _ = pressure.gl_nodes_weights(N - 1)
    I, Dg, _ = pressure.interpolation_matrices(N)
    for d in range(N + 1):
        np.testing.assert_allclose(I @ xi ** d, zeta ** d, rtol=0, atol=1e-13)
        deriv = d * zeta ** (d - 1) if d else np.zeros_like(zeta)
        np.testing.assert_allclose(Dg @ xi ** d, deriv, rtol=0, atol=1e-11 * max(1, d))


def _gl_coords(m_, N):
    I, _, _ = pressure.interpolation_matrices(N)
    return np.stack([pressure._contract(I, I, I, m_.xyz[:, c]) for c in range(3)])  # [3, E, m, m, m]


def _monomial_integral(p, L):
    return L ** (p + 1) / (p + 1)


@pytest.mark.parametrize("N", [3, 4])
def test_weak_divergence_is_exact_quadrature_on_affine_box(N):
    """For u_a of degree <= N-1 and psi of degree <= N-2 in each coordinate, GL
    quadrature is exact on axis-aligned affine elements: sum_q psi(x_q) (D_a u_a)_q
    = int psi d(u_a)/dx_a dx, taken here in closed form from the monomials."""
    lx, ly, lz = 1.0, 2.0, 3.5
    m_ = mesh.box(2, 3, 1, N, lx, ly, lz)
    F, _ = pressure.div_factors(m_)
    X = m_.xyz
    Xg = _gl_coords(m_, N)
    rng = np.random.default_rng(7)
    for a in range(3):
        for _ in range(3):
            e_u = rng.integers(0, N, size=3)       # degree <= N-1 per coordinate
            e_p = rng.integers(0, N - 1, size=3)   # degree <= N-2
            e_u[a] = max(e_u[a], 1)
            u = np.zeros((3, m_.E) + (N + 1,) * 3)
            u[a] = X[:, 0] ** e_u[0] * X[:, 1] ** e_u[1] * X[:, 2] ** e_u[2]
            psi = Xg[0] ** e_p[0] * Xg[1] ** e_p[1] * Xg[2] ** e_p[2]
            got = np.sum(psi * pressure.div_local(N, F, u))
            L = (lx, ly, lz)
            exact = float(e_u[a])
            for c in range(3):
                pw = e_p[c] + e_u[c] - (1 if c == a else 0)
                exact *= _monomial_integral(pw, L[c])
            assert abs(got - exact) <= 1e-12 * max(1.0, abs(exact)), (a, e_u, e_p, got, exact)


def test_divergence_of_coordinates_is_gl_volume_on_curved_pipe():
    """The coordinates are in the isoparametric space, so div(x, 0, 0) at a GL
    point is rho^3 sum_b adj(J)_{b0} J_{0b} = rho^3 det(J), and div(y, 0, 0) is 0
    (adj(J) J = det(J) I).  A transposed adjugate fails this on curved elements."""
    N = 5
    m_ = mesh.pipe(2, 2, 2, N, L=2.0)
    F, det = pressure.div_factors(m_)
    _, _, rho = pressure.interpolation_matrices(N)
    rho3 = rho[:, None, None] * rho[None, :, None] * rho[None, None, :]
    vol = rho3 * det
    for a in range(3):
        for c in range(3):
            u = np.zeros((3, m_.E) + (N + 1,) * 3)
            u[a] = m_.xyz[:, c]
            d = pressure.div_local(N, F, u)
            if a == c:
                np.testing.assert_allclose(d, vol, rtol=1e-13, atol=0)
            else:
                assert np.abs(d).max() < 1e-13 * vol.max()
    # the GL quadrature of the volume converges to pi R^2 L
    assert abs(vol.sum() - np.pi * 2.0) < 1e-2


@pytest.mark.parametrize("N", [2, 3, 4])
def test_affine_element_matches_kronecker_divergence(N):
    """On one axis-aligned element of size hx x hy x hz: F[b, a] = 0 for b != a and
    D_0 = (hy hz / 4) diag(rho (x) rho (x) rho) (I (x) I (x) Dg) (k factor leftmost)."""
    hx, hy, hz = 0.5, 2.0 / 3.0, 3.5
    m_ = mesh.box(1, 1, 1, N, hx, hy, hz)
    F, _ = pressure.div_factors(m_)
    I, Dg, rho = pressure.interpolation_matrices(N)
    R3 = np.diag(np.kron(rho, np.kron(rho, rho)))
    kron3 = lambda a, b, c: np.kron(a, np.kron(b, c))  # noqa: E731
    K = [(hy * hz / 4) * R3 @ kron3(I, I, Dg),
         (hx * hz / 4) * R3 @ kron3(I, Dg, I),
         (hx * hy / 4) * R3 @ kron3(Dg, I, I)]
    n3 = (N + 1) ** 3
    for a in range(3):
        cols = []
        for q in range(n3):
            u = np.zeros((3, 1) + (N + 1,) * 3)
            u[a].reshape(-1)[q] = 1.0
            cols.append(pressure.div_local(N, F, u).reshape(-1))
        A = np.array(cols).T
        assert np.abs(A - K[a]).max() <= 1e-14 * np.abs(K[a]).max()


def test_gradient_is_the_transpose_of_divergence():
    N = 5
    m_ = mesh.pipe(2, 1, 2, N, L=1.5)
    F, _ = pressure.div_factors(m_)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((3, m_.E) + (N + 1,) * 3)
    p = rng.standard_normal((m_.E,) + (N - 1,) * 3)
    lhs = np.sum(p * pressure.div_local(N, F, u))
    rhs = np.sum(pressure.grad_local(N, F, p) * u)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs) * 10


def test_consistent_poisson_operator_has_only_the_constant_null_mode():
    """Box with Dirichlet velocity on every face, N = 4: E is symmetric positive
    semi-definite; constants span its null space (GL quadrature is exact for the
    weak gradient of a constant on affine elements when N >= 3), and there is no
    other (spurious) zero mode -- the point of the staggered pair."""
    m_ = mesh.box(2, 2, 2, 4)
    P = pressure.Pressure(solver.Problem(m_))
    A = P.dense()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    ones = np.ones(P.shape)
    assert np.abs(P.E(ones)).max() < 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[0] > -1e-13 * ev[-1]
    assert abs(ev[0]) < 1e-13 * ev[-1]
    assert ev[1] > 1e-4 * ev[-1]


def test_operator_symmetry_on_curved_pipe():
    m_ = mesh.pipe(2, 1, 2, 4, L=1.0)
    P = pressure.Pressure(solver.Problem(m_))
    p = vectors.local_field(11, m_.E, 3)
    q = vectors.local_field(12, m_.E, 3)
    a, b = np.sum(q * P.E(p)), np.sum(p * P.E(q))
    assert abs(a - b) < 1e-13 * abs(a) * 10
    assert np.sum(p * P.E(p)) > 0


@pytest.mark.parametrize("maker", [lambda: mesh.box(2, 2, 2, 4), lambda: mesh.pipe(2, 1, 3, 3, L=1.5)])
def test_pressure_cg_matches_dense_solve_on_the_mean_free_space(maker):
    """CG on Pm E Pm against the dense minimum-norm solution (eigendecomposition
    of the projected matrix, its one zero mode dropped)."""
    P = pressure.Pressure(solver.Problem(maker()))
    g = vectors.local_field(21, P.shape[0], P.shape[1])
    x, it, rel, st = pressure.cg(P, g, tol=1e-12)
    assert st == solver.CONVERGED and rel <= 1e-12
    A = P.dense()
    n = A.shape[0]
    Pm = np.eye(n) - np.ones((n, n)) / n
    S = Pm @ A @ Pm
    ev, V = np.linalg.eigh(0.5 * (S + S.T))
    assert abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 1e-6 * ev[-1]  # one zero mode: the constant
    gv = Pm @ g.reshape(-1)
    xd = V[:, 1:] @ ((V[:, 1:].T @ gv) / ev[1:])
    assert np.linalg.norm(x.reshape(-1) - xd) <= 1e-9 * np.linalg.norm(xd)
    assert abs(x.sum()) <= 1e-10 * np.abs(x).sum()
    # Pm (g - E x) = 0: the residual of the unprojected equation is a constant
    res = g - P.E(x)
    assert np.abs(res - res.mean()).max() <= 1e-9 * np.abs(g).max()


def test_pressure_cg_zero_rhs_and_constant_rhs():
    P = pressure.Pressure(solver.Problem(mesh.box(2, 1, 1, 3)))
    for g in (np.zeros(P.shape), np.full(P.shape, 2.5)):
        x, it, rel, st = pressure.cg(P, g)
        assert st == solver.CONVERGED and it == 0 and not x.any()


@pytest.mark.parametrize("kind,N", [("box", 2), ("box", 3), ("box", 4), ("pipe", 3), ("pipe_open", 4)])
def test_diagonal_is_the_dense_diagonal(kind, N):
    """Pressure.diagonal() (the Jacobi preconditioner, rows of the weak
    divergence squared against mask / assembled mass) against the diagonal
    of E assembled column by column from unit pressures."""
    if kind == "box":
        m_ = mesh.box(2, 1, 2, N, lx=1.0, ly=0.7, lz=1.3)
    elif kind == "pipe":
        m_ = mesh.pipe(1, 1, 3, N, L=1.5)
    else:
        m_ = mesh.pipe(1, 1, 3, N, L=1.5, periodic=False)
    P = pressure.Pressure(solver.Problem(m_))
    d = P.diagonal()
    assert np.all(d > 0)
    np.testing.assert_allclose(d.reshape(-1), np.diag(P.dense()), rtol=1e-13, atol=0)


def test_jacobi_cg_reaches_the_plain_solution_in_fewer_iterations():
    m_ = mesh.pipe(2, 1, 3, 4, L=1.5)
    P = pressure.Pressure(solver.Problem(m_))
    g = np.random.default_rng(5).standard_normal(P.shape)
    x0, it0, r0, s0 = pressure.cg(P, g, tol=1e-10)
    x1, it1, r1, s1 = pressure.cg(P, g, tol=1e-10, dinv=1.0 / P.diagonal())
    assert s0 == solver.CONVERGED and s1 == solver.CONVERGED
    assert r1 <= 1e-10 and it1 < it0
    assert abs(x1.mean()) <= 1e-12 * np.abs(x1).max()
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-7 * np.abs(x0).max())


@pytest.mark.parametrize("jacobi", [False, True])
def test_pressure_cg_iterates_minimise_the_energy_error_over_the_krylov_space(jacobi):
    """On the mean-free space the pressure CG is CG for S = Pm E Pm with the
    preconditioner Pm D^-1 Pm (Jacobi) or Pm: its k-th iterate is the
    S-norm-closest element of K_k(M S, M Pm g), computed densely (Arnoldi on
    the dense E), so a wrong projection, step or direction update fails."""
    P = pressure.Pressure(solver.Problem(mesh.pipe(2, 1, 3, 3, L=1.5)))
    A = P.dense()
    n = A.shape[0]
    Pm = np.eye(n) - np.ones((n, n)) / n
    S = Pm @ A @ Pm
    dinv = 1.0 / P.diagonal()
    M = Pm @ np.diag(dinv.reshape(-1)) @ Pm if jacobi else Pm
    g = vectors.local_field(31, P.shape[0], P.shape[1])
    gv = Pm @ g.reshape(-1)
    Q = []
    v = M @ gv
    for k in range(1, 7):
        for _ in range(2):
            for q in Q:
                v = v - (q @ v) * q
        Q.append(v / np.linalg.norm(v))
        V = np.stack(Q, axis=1)
        ref = V @ np.linalg.solve(V.T @ S @ V, V.T @ gv)
        x, it, rel, st = pressure.cg(P, g, tol=1e-30, maxit=k, dinv=dinv if jacobi else None)
        assert it == k
        assert np.linalg.norm(x.reshape(-1) - ref) <= 1e-9 * np.linalg.norm(ref), k
        v = M @ (S @ Q[-1])
