"""Pins for the oracle's meshes and geometric factors g1..g6, B (Alg. 1 inputs)."""

import numpy as np
import pytest

from oracle import geometry, gll, mesh


def test_affine_box_factors_closed_form():
    # Distinct element sizes per axis so that a swapped axis or factor shows.
    N, nx, ny, nz, lx, ly, lz = 4, 2, 3, 1, 1.0, 2.0, 3.5
    m = mesh.box(nx, ny, nz, N, lx, ly, lz)
    G, B, detJ = geometry.factors(m)
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    _, w = gll.nodes_weights(N)
    w3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()  # noqa: E731
    assert rel(G[:, 0], np.broadcast_to(w3 * hy * hz / (2 * hx), G[:, 0].shape)) < 1e-14
    assert rel(G[:, 1], np.broadcast_to(w3 * hx * hz / (2 * hy), G[:, 1].shape)) < 1e-14
    assert rel(G[:, 2], np.broadcast_to(w3 * hx * hy / (2 * hz), G[:, 2].shape)) < 1e-14
    assert np.abs(G[:, 3:]).max() < 1e-14 * np.abs(G[:, :3]).max()
    assert rel(B, np.broadcast_to(w3 * hx * hy * hz / 8, B.shape)) < 1e-14
    assert abs(B.sum() - lx * ly * lz) < 1e-13


def test_sheared_element_factors():
    # x = A r + c on one element: J = A, G = w3 det(A) A^{-1} A^{-T} (cofactor form).
    N = 3
    A = np.array([[0.7, 0.2, 0.1], [-0.1, 0.9, 0.3], [0.05, -0.2, 1.1]])
    x, w = gll.nodes_weights(N)
    r = np.stack(np.meshgrid(x, x, x, indexing="ij")[::-1])  # [3 (r,s,t), k, j, i]
    xyz = np.einsum("ab,bkji->akji", A, r)[None] + np.array([0.3, -1.0, 2.0])[None, :, None, None, None]
    m = mesh.Mesh(N, xyz, np.zeros((1, 6), bool))
    G, B, detJ = geometry.factors(m)
    # adjugate written out by cofactors (independent of numpy.linalg)
    cof = np.array([[A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1], -(A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0]), A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0]],
                    [-(A[0, 1] * A[2, 2] - A[0, 2] * A[2, 1]), A[0, 0] * A[2, 2] - A[0, 2] * A[2, 0], -(A[0, 0] * A[2, 1] - A[0, 1] * A[2, 0])],
                    [A[0, 1] * A[1, 2] - A[0, 2] * A[1, 1], -(A[0, 0] * A[1, 2] - A[0, 2] * A[1, 0]), A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]]])
    det = A[0, 0] * cof[0, 0] + A[0, 1] * cof[0, 1] + A[0, 2] * cof[0, 2]
    Ainv = cof.T / det  # Ainv[b, a] = d r_b / d x_a
    M = det * Ainv @ Ainv.T
    w3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for c, (p, q) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        np.testing.assert_allclose(G[0, c], w3 * M[p, q], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(B[0], w3 * det, rtol=1e-13)


@pytest.mark.parametrize("periodic", [True, False])
def test_pipe_positive_jacobian_and_volume_convergence(periodic):
    errs = []
    for N in (2, 4, 6, 8):
        m = mesh.pipe(2, 2, 2, N, R=1.0, L=2.0, periodic=periodic)
        G, B, detJ = geometry.factors(m)
        assert detJ.min() > 0
        errs.append(abs(B.sum() - np.pi * 2.0) / (np.pi * 2.0))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-6, errs


def test_pipe_wall_points_on_circle():
    m = mesh.pipe(4, 2, 1, 5, R=1.5, L=1.0)
    wallpts = m.xyz[m.dirichlet_face[:, 1]][:, :, :, :, -1]  # i = N face
    r = np.hypot(wallpts[:, 0], wallpts[:, 1])
    np.testing.assert_allclose(r, 1.5, rtol=0, atol=1e-14)


def test_element_counts():
    assert mesh.pipe(8, 2, 4, 1).E == 8 * (8 + 8) * 4
    assert mesh.box(3, 2, 5, 1).E == 30
