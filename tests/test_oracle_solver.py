"""Pins for the oracle's assembled operator, Jacobi diagonal and PCG (Sec. 2)."""

import numpy as np
import pytest

from oracle import mesh, solver
from sem_inputs import forcing


@pytest.mark.parametrize("maker,h2", [
    (lambda: mesh.box(2, 2, 2, 3), 0.0),
    (lambda: mesh.pipe(2, 1, 2, 3, L=2.0), 0.0),
    (lambda: mesh.pipe(2, 1, 2, 2, L=2.0), 5.0),
])
def test_dense_spd_pcg_matches_cholesky(maker, h2):
    m = maker()
    P = solver.Problem(m, 1.0, h2)
    A, free, rep = P.dense()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    L = np.linalg.cholesky(A)  # raises unless SPD
    assert L.shape == A.shape
    # Jacobi diagonal equals the dense diagonal
    Minv = P.jacobi_inverse().reshape(-1)
    np.testing.assert_allclose(1.0 / Minv[rep[free]], np.diag(A), rtol=1e-13)
    # PCG vs a direct solve
    f = forcing.evaluate(m.xyz, forcing.random_modes(7, L=2.0))
    b = P.rhs(f)
    res = solver.pcg(P, b)
    assert res.status == solver.CONVERGED and res.rel_res <= 1e-10
    xd = np.linalg.solve(A, b.reshape(-1)[rep[free]])
    xg = res.x.reshape(-1)[rep[free]]
    assert np.linalg.norm(xg - xd) <= 1e-9 * np.linalg.norm(xd)


def krylov_optima(A, prec, bg, kmax):
    """(k, x_k) for k = 1..kmax: the A-norm-closest element to A^-1 bg of the
    preconditioned Krylov space K_k(M A, M bg), x_k = V (V^T A V)^-1 V^T bg,
    with V built by Arnoldi (modified Gram-Schmidt, twice) on the dense
    matrix; prec(v) applies M."""
    Q = []
    v = prec(bg)
    for k in range(1, kmax + 1):
        for _ in range(2):
            for q in Q:
                v = v - (q @ v) * q
        Q.append(v / np.linalg.norm(v))
        V = np.stack(Q, axis=1)
        yield k, V @ np.linalg.solve(V.T @ A @ V, V.T @ bg)
        v = prec(A @ Q[-1])


@pytest.mark.parametrize("maker,h2", [
    (lambda: mesh.pipe(2, 1, 2, 3, L=2.0), 0.0),
    (lambda: mesh.box(2, 2, 2, 3), 1.5),
])
def test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space(maker, h2):
    """k steps of Jacobi-PCG from x0 = 0 give the element of the Krylov space
    K_k(M^-1 A, M^-1 b) closest to the solution in the A-norm (Hestenes and
    Stiefel 1952): x_k = V (V^T A V)^-1 V^T b for any basis V of that space.
    V is built by Arnoldi on the dense matrix, independently of the oracle's
    recurrences, so a wrong step length, direction update, inner product or
    preconditioner application fails at some k."""
    m = maker()
    P = solver.Problem(m, 1.0, h2)
    A, free, rep = P.dense()
    minv = P.jacobi_inverse().reshape(-1)[rep[free]]
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(11, L=2.0)))
    bg = b.reshape(-1)[rep[free]]
    for k, ref in krylov_optima(A, lambda v: minv * v, bg, 7):
        res = solver.pcg(P, b, tol=1e-30, maxit=k)
        got = res.x.reshape(-1)[rep[free]]
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), k


def test_fp32_inner_pcg_iterates_follow_the_krylov_optimum():
    """The FP32 inner PCG of the mixed solvers is the same CG in single
    precision: its k-th iterate matches the FP64 Krylov optimum to FP32
    accuracy."""
    m = mesh.pipe(2, 1, 2, 3, L=2.0)
    P = solver.Problem(m)
    A, free, rep = P.dense()
    minv = P.jacobi_inverse().reshape(-1)[rep[free]]
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(11, L=2.0)))
    bg = b.reshape(-1)[rep[free]]
    p32 = solver.Problem32(P)
    for k, ref in krylov_optima(A, lambda v: minv * v, bg, 6):
        x32, it, st = solver.pcg32(p32, b.astype(np.float32), 1e-30, k)
        assert it == k
        got = x32.astype(np.float64).reshape(-1)[rep[free]]
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), k


@pytest.mark.parametrize("delta", [0.0, 0.9])
def test_reliable_updates_keep_the_krylov_iterates(delta):
    """The reliable-update solver replaces the FP32 recurrence residual by the
    FP64 true one and keeps CG's direction (Sleijpen and van der Vorst 1996),
    so its iterates stay the Krylov optimum of the FP64 problem, to FP32
    accuracy, whether it never replaces (delta = 0) or replaces after every
    iteration (delta = 0.9).  A solver that restarted CG at a replacement, or
    mixed up the scaling of its increment, leaves that optimum."""
    m = mesh.pipe(2, 1, 2, 3, L=2.0)
    P = solver.Problem(m)
    A, free, rep = P.dense()
    minv = P.jacobi_inverse().reshape(-1)[rep[free]]
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(11, L=2.0)))
    bg = b.reshape(-1)[rep[free]]
    for k, ref in krylov_optima(A, lambda v: minv * v, bg, 8):
        res = solver.pcg_mixed_reliable(P, b, tol=1e-30, delta=delta, maxit=k)
        assert res.outer_iters == (k if delta > 0 else 0)
        got = res.x.reshape(-1)[rep[free]]
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), k


def test_manufactured_solution_spectral_convergence_box():
    errs = []
    for N in (2, 4, 6, 8):
        m = mesh.box(2, 2, 2, N)
        P = solver.Problem(m)
        b = P.rhs(forcing.manufactured(m.xyz))
        res = solver.pcg(P, b, tol=1e-13)
        errs.append(np.abs(res.x - forcing.manufactured_solution(m.xyz)).max())
    assert all(errs[i + 1] < 0.05 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-6, errs


def test_manufactured_solution_converges_on_curved_pipe():
    # u* = (1 - r^2) cos(2 pi z / L): zero on the wall r = 1, periodic in z;
    # f = -lap u* = [4 + (1 - r^2) (2 pi / L)^2] cos(2 pi z / L).
    L = 2.0
    k = 2 * np.pi / L
    errs = []
    for N in (3, 5, 7):
        m = mesh.pipe(2, 1, 2, N, L=L)
        x, y, z = m.xyz[:, 0], m.xyz[:, 1], m.xyz[:, 2]
        r2 = x * x + y * y
        f = (4.0 + (1.0 - r2) * k * k) * np.cos(k * z)
        ustar = (1.0 - r2) * np.cos(k * z)
        P = solver.Problem(m)
        res = solver.pcg(P, P.rhs(f), tol=1e-13)
        errs.append(np.abs(res.x - ustar).max())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[-1] < 1e-4, errs


def test_zero_rhs_and_initial_guess():
    m = mesh.box(2, 2, 2, 3)
    P = solver.Problem(m)
    res = solver.pcg(P, np.zeros(P.shape))
    assert res.iters == 0 and np.all(res.x == 0)
    b = P.rhs(forcing.manufactured(m.xyz))
    exact = solver.pcg(P, b, tol=1e-13).x
    res = solver.pcg(P, b, x0=exact)
    assert res.iters == 0


@pytest.mark.parametrize("inner_tol", [1e-3, 1e-5])
def test_mixed_precision_refinement(inner_tol):
    m = mesh.pipe(2, 1, 2, 4, L=2.0)
    P = solver.Problem(m, 1.0, 0.5)
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(3, L=2.0)))
    res = solver.pcg_mixed(P, b, tol=1e-10, inner_tol=inner_tol)
    assert res.status == solver.CONVERGED
    r = b - P.A(res.x)
    assert np.sqrt(P.dot(r, r) / P.dot(b, b)) <= 1e-10
    ref = solver.pcg(P, b, tol=1e-12).x
    err = np.sqrt(P.dot(res.x - ref, res.x - ref) / P.dot(ref, ref))
    assert err < 1e-8
    assert res.outer_iters >= 2  # FP32 alone cannot reach 1e-10


def test_mixed_reliable_updates():
    m = mesh.pipe(2, 1, 3, 5, L=2.0)
    P = solver.Problem(m, 1.0, 0.3)
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(4, L=2.0)))
    ref = solver.pcg(P, b, tol=1e-10)
    res = solver.pcg_mixed_reliable(P, b, tol=1e-10)
    assert res.status == solver.CONVERGED
    r = b - P.A(res.x)
    assert np.sqrt(P.dot(r, r) / P.dot(b, b)) <= 1e-10
    # keeping the Krylov direction: close to the FP64 iteration count, far
    # below restarted refinement
    assert res.iters <= 1.25 * ref.iters + 5, (res.iters, ref.iters)
    restarted = solver.pcg_mixed(P, b, tol=1e-10, inner_tol=1e-4)
    assert res.iters < restarted.iters
    assert res.outer_iters >= 2
    err = np.sqrt(P.dot(res.x - ref.x, res.x - ref.x) / P.dot(ref.x, ref.x))
    assert err < 1e-8
