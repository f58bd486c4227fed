"""Pins for the oracle's overlapping Schwarz preconditioner (Sec. 2, Eq. 6):
fast-diagonalisation local solves and the trilinear coarse grid."""

import numpy as np
import pytest

from oracle import gll, mesh, schwarz, solver


def tensor_box(bx, by, bz, N):
    """Axis-aligned box with element breakpoints bx, by, bz (unequal element
    sizes), element e = ex + nx (ey + ny ez), Dirichlet on all six faces."""
    xi, _ = gll.nodes_weights(N)
    nx, ny, nz = len(bx) - 1, len(by) - 1, len(bz) - 1
    n = N + 1
    E = nx * ny * nz
    xyz = np.empty((E, 3, n, n, n))
    dface = np.zeros((E, 6), dtype=bool)
    seg = lambda b, k: b[k] * (1 - xi) / 2 + b[k + 1] * (1 + xi) / 2  # noqa: E731
    for e in range(E):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        xyz[e, 0] = seg(bx, ex)[None, None, :]
        xyz[e, 1] = seg(by, ey)[None, :, None]
        xyz[e, 2] = seg(bz, ez)[:, None, None]
        dface[e] = [ex == 0, ex == nx - 1, ey == 0, ey == ny - 1, ez == 0, ez == nz - 1]
    return mesh.Mesh(N, xyz, dface, None, "box")


@pytest.mark.parametrize("h2", [0.0, 2.5])
def test_fdm_local_solve_is_the_exact_overlapping_subdomain_inverse_on_a_tensor_box(h2):
    """On an axis-aligned box the assembled operator is a sum of Kronecker
    products of assembled 1D operators, so the separable local operator equals
    R_e A R_e^T (the principal submatrix on the element's free nodes, which
    holds the neighbours' contributions at the shared nodes) exactly.  Unequal
    element sizes make a wrong neighbour length or a swapped end fail."""
    N = 3
    m_ = tensor_box([0.0, 0.3, 1.0, 1.2], [0.0, 0.5, 0.7], [0.0, 0.4, 1.1], N)
    prob = solver.Problem(m_, 1.0, h2)
    sw = schwarz.Schwarz(prob, coarse=False)
    A, free, _ = prob.dense()
    pos = {int(g): c for c, g in enumerate(free)}
    glo = prob.glo.reshape(prob.shape)
    mask = prob.mask
    for e in range(m_.E):
        loc = np.flatnonzero(mask[e].reshape(-1) > 0)
        idx = [pos[int(g)] for g in glo[e].reshape(-1)[loc]]
        ref = np.linalg.inv(A[np.ix_(idx, idx)])
        got = np.empty_like(ref)
        for c, q in enumerate(loc):
            r = np.zeros(prob.shape)
            r[e].reshape(-1)[q] = 1.0
            got[:, c] = sw.local_solve(r)[e].reshape(-1)[loc]
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), e


def test_coarse_functions_reproduce_trilinear_fields():
    """The eight vertex functions are a partition of unity, each is 1 at its
    own vertex, and together they reproduce the (affine) coordinates."""
    m_ = tensor_box([0.0, 0.3, 1.0], [0.0, 0.5, 0.7], [0.0, 0.4], 4)
    sw = schwarz.Schwarz(solver.Problem(m_), coarse=True)
    phi = sw._phi
    np.testing.assert_allclose(phi.sum(axis=0), 1.0, rtol=0, atol=1e-15)
    N = m_.N
    for v in range(8):
        c = (N * ((v >> 2) & 1), N * ((v >> 1) & 1), N * (v & 1))
        assert phi[v][c] == 1.0
        for e in range(m_.E):
            for a in range(3):
                xv = np.array([m_.xyz[e, a][(N * ((u >> 2) & 1), N * ((u >> 1) & 1), N * (u & 1))] for u in range(8)])
                np.testing.assert_allclose(np.einsum("v,vkji->kji", xv, phi), m_.xyz[e, a], rtol=0, atol=1e-14)


@pytest.mark.parametrize("maker", [lambda: mesh.box(2, 2, 2, 3), lambda: mesh.pipe(2, 1, 3, 3, L=1.5)])
@pytest.mark.parametrize("coarse", [False, True])
def test_preconditioner_is_symmetric_positive_definite(maker, coarse):
    prob = solver.Problem(maker())
    sw = schwarz.Schwarz(prob, coarse=coarse)
    A, free, rep = prob.dense()
    glo = prob.glo.reshape(prob.shape)
    M = np.zeros_like(A)
    for c, g in enumerate(free):
        r = (glo == g).astype(np.float64)
        z = sw.apply(r)
        # z is a continuous field (equal on every copy of a node) and zero on
        # the Dirichlet nodes, like the CG vectors it feeds
        assert np.abs(z[prob.mask == 0]).max(initial=0.0) == 0.0
        np.testing.assert_allclose(prob.gs(z / prob.mult), z, rtol=0, atol=1e-13 * np.abs(z).max())
        M[:, c] = z.reshape(-1)[rep[free]]
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T))[0] > 0


def test_schwarz_pcg_iterates_minimise_the_energy_error_over_the_krylov_space():
    """Schwarz-PCG is CG with z = M r: its k-th iterate is the A-norm-closest
    element of K_k(M A, M b), computed densely (M assembled column by column
    from the preconditioner, the space by Arnoldi)."""
    prob = solver.Problem(mesh.pipe(2, 1, 3, 3, L=1.5))
    sw = schwarz.Schwarz(prob, coarse=True)
    A, free, rep = prob.dense()
    glo = prob.glo.reshape(prob.shape)
    M = np.zeros_like(A)
    for c, g in enumerate(free):
        M[:, c] = sw.apply((glo == g).astype(np.float64)).reshape(-1)[rep[free]]
    b = prob.rhs(np.random.default_rng(1).standard_normal(prob.shape))
    bg = b.reshape(-1)[rep[free]]
    Q = []
    v = M @ bg
    for k in range(1, 7):
        for _ in range(2):
            for q in Q:
                v = v - (q @ v) * q
        Q.append(v / np.linalg.norm(v))
        V = np.stack(Q, axis=1)
        ref = V @ np.linalg.solve(V.T @ A @ V, V.T @ bg)
        res = schwarz.pcg(prob, b, sw.apply, tol=1e-30, maxit=k)
        got = res.x.reshape(-1)[rep[free]]
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), k
        v = M @ (A @ Q[-1])


def test_schwarz_pcg_solves_the_system_and_the_coarse_grid_bounds_iterations():
    """Schwarz-PCG reaches the same solution as Jacobi-PCG.  With the coarse
    grid its iteration count stays flat as the pipe grows from 3 to 12 layers
    (Jacobi's and the local-solves-only count grow)."""
    its = {}
    for nzp in (3, 12):
        prob = solver.Problem(mesh.pipe(2, 1, nzp, 4, L=nzp / 2.0))
        b = prob.rhs(np.random.default_rng(1).standard_normal(prob.shape))
        rj = solver.pcg(prob, b)
        rs = schwarz.pcg(prob, b, schwarz.Schwarz(prob, coarse=True).apply)
        assert rs.status == solver.CONVERGED
        err = np.sqrt(prob.dot(rs.x - rj.x, rs.x - rj.x) / prob.dot(rj.x, rj.x))
        assert err <= 1e-8
        r_true = b - prob.A(rs.x)
        assert np.sqrt(prob.dot(r_true, r_true) / prob.dot(b, b)) <= 1.1e-10
        its[nzp] = (rj.iters, rs.iters)
    (j3, s3), (j12, s12) = its[3], its[12]
    assert s3 <= j3 / 3 and s12 <= j12 / 4
    assert s12 <= s3 + 4
