"""Pins of the oracle's projection onto previous solutions (oracle/projection.py)
against facts that do not depend on it: the dense A-orthogonal projection
written with a linear solve, exact reproduction of right-hand sides inside the
span, A-orthonormality, and the restart rule."""

import numpy as np
import pytest

from oracle import mesh as omesh, projection, solver
from sem_inputs import forcing

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _problem(h2=0.0):
    return solver.Problem(omesh.pipe(2, 1, 3, 3, L=2.0), 1.0, h2)


def _rhs(P, seed):
    return P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(seed, L=2.0)))


def test_basis_is_a_orthonormal():
    P = _problem()
    proj = projection.Projection(P, 8)
    for s in range(5):
        proj.solve(_rhs(P, 20 + s), tol=1e-11)
    X, AX = proj.X, proj.AX
    G = np.array([[P.dot(x, ay) for ay in AX] for x in X])
    assert G.shape == (5, 5)
    assert np.abs(G - np.eye(5)).max() < 1e-10
    # AX really is A X
    for x, ax in zip(X, AX):
        assert np.linalg.norm(P.A(x) - ax) <= 1e-12 * np.linalg.norm(ax)


def test_guess_is_the_dense_a_orthogonal_projection():
    """xbar = S (S^T A S)^{-1} S^T b for S = the earlier solutions, with the
    dense assembled matrix."""
    P = _problem(h2=0.7)
    A, free, rep = P.dense()
    proj = projection.Projection(P, 8)
    sols = []
    for s in range(3):
        sols.append(proj.solve(_rhs(P, 40 + s), tol=1e-12).x)
    b = _rhs(P, 99)
    xbar, _ = proj.guess(b)
    S = np.stack([x.reshape(-1)[rep[free]] for x in sols], axis=1)
    bg = b.reshape(-1)[rep[free]]
    ref = S @ np.linalg.solve(S.T @ A @ S, S.T @ bg)
    got = xbar.reshape(-1)[rep[free]]
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_right_hand_sides_in_the_span_need_no_iterations():
    P = _problem()
    proj = projection.Projection(P, 8)
    bs = [_rhs(P, 60 + s) for s in range(3)]
    xs = [proj.solve(b, tol=1e-12).x for b in bs]
    again = proj.solve(bs[1], tol=1e-9)
    assert again.iters == 0
    assert np.linalg.norm(again.x - xs[1]) <= 1e-9 * np.linalg.norm(xs[1])
    combo = proj.solve(2.0 * bs[0] - 0.5 * bs[2], tol=1e-9)
    assert combo.iters == 0
    # without a basis the same solve takes many iterations
    assert solver.pcg(P, 2.0 * bs[0] - 0.5 * bs[2], tol=1e-9).iters > 10


def test_full_basis_restarts_from_the_newest_solution():
    P = _problem()
    proj = projection.Projection(P, 2)
    res = [proj.solve(_rhs(P, 80 + s), tol=1e-11) for s in range(3)]
    assert len(proj.X) == 1
    x = res[-1].x
    x_a = x / np.sqrt(P.dot(x, P.A(x)))
    assert np.linalg.norm(proj.X[0] - x_a) <= 1e-12 * np.linalg.norm(x_a)


def test_slowly_varying_sequence_takes_fewer_iterations():
    P = _problem()
    base = forcing.random_modes(5, L=2.0)
    proj = projection.Projection(P, 8)
    with_p, without = 0, 0
    for k in range(6):
        f = forcing.evaluate(P.mesh.xyz, base) * (1.0 + 0.05 * k) + 0.01 * k * P.mesh.xyz[:, 2]
        b = P.rhs(f)
        with_p += proj.solve(b, tol=1e-10).iters
        without += solver.pcg(P, b, tol=1e-10).iters
    assert with_p < 0.5 * without
