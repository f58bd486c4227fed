"""Pins for the oracle's local operator (Alg. 1 + the h2 mass term of Sec. 2, Eq. 4)."""

import numpy as np
import pytest

from oracle import geometry, gll, mesh, numbering, operator
from sem_inputs import vectors


def _apply_to_units(G, B, D, h1, h2, e=0):
    n = D.shape[0]
    cols = []
    for q in range(n ** 3):
        u = np.zeros((1, n, n, n))
        u.reshape(-1)[q] = 1.0
        cols.append(operator.ax_local(u, G[e:e + 1], B[e:e + 1], D, h1, h2).reshape(-1))
    return np.array(cols).T


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.3, 2.5)])
def test_affine_element_matches_kronecker_matrix(N, h1, h2):
    hx, hy, hz = 0.5, 2.0 / 3.0, 3.5
    m = mesh.box(2, 3, 1, N, 1.0, 2.0, 3.5)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(N)
    A = _apply_to_units(G, B, D, h1, h2)
    K = operator.element_matrix_affine(N, hx, hy, hz, h1, h2)
    assert np.abs(A - K).max() <= 1e-13 * np.abs(K).max()


def test_constants_in_kernel_and_symmetry_on_curved_pipe():
    m = mesh.pipe(2, 2, 2, 5, L=2.0)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(5)
    ones = np.ones((m.E, 6, 6, 6))
    w = operator.ax_local(ones, G, B, D, 1.0, 0.0)
    assert np.abs(w).max() < 1e-13 * np.abs(G).max() * 36
    u = vectors.local_field(1, m.E, 6)
    v = vectors.local_field(2, m.E, 6)
    for h1, h2 in [(1.0, 0.0), (0.7, 3.0)]:
        Au = operator.ax_local(u, G, B, D, h1, h2)
        Av = operator.ax_local(v, G, B, D, h1, h2)
        lhs = np.einsum("ekji,ekji->e", u, Av)
        rhs = np.einsum("ekji,ekji->e", v, Au)
        assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()
        # positive semi-definite per element
        assert np.einsum("ekji,ekji->e", u, Au).min() > 0


def test_local_diagonal_matches_unit_vectors_on_curved_element():
    m = mesh.pipe(2, 1, 1, 3, L=1.0)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(3)
    e = m.E - 1  # an outer, curved ring element
    A = _apply_to_units(G, B, D, 0.6, 1.7, e)
    diag = operator.local_diagonal(G, B, D, 0.6, 1.7)[e].reshape(-1)
    np.testing.assert_allclose(diag, np.diag(A), rtol=1e-13, atol=0)


def _trilinear_box(nx, ny, nz, N, seed, amp=0.15):
    """Box whose interior vertices are moved at random; every element is the
    trilinear map of its 8 vertices evaluated at the GLL points."""
    x, _ = gll.nodes_weights(N)
    rng = np.random.default_rng(seed)
    V = np.stack(np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny,
                             np.arange(nz + 1) / nz, indexing="ij"), axis=-1)
    inner = (slice(1, nx), slice(1, ny), slice(1, nz))
    V[inner] += amp * rng.uniform(-1, 1, V[inner].shape) / max(nx, ny, nz)
    n = N + 1
    lo, hi = (1 - x) / 2, (1 + x) / 2
    xyz = np.empty((nx * ny * nz, 3, n, n, n))
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                e = ex + nx * (ey + ny * ez)
                acc = 0.0
                for c in range(8):
                    a, b, d = c & 1, (c >> 1) & 1, (c >> 2) & 1
                    wi = (hi if a else lo)[None, None, :]
                    wj = (hi if b else lo)[None, :, None]
                    wk = (hi if d else lo)[:, None, None]
                    acc = acc + (wk * wj * wi)[None] * V[ex + a, ey + b, ez + d][:, None, None, None]
                xyz[e] = acc
    return mesh.Mesh(N, xyz, mesh.box(nx, ny, nz, N).dirichlet_face)


def test_patch_test_on_trilinear_mesh():
    # Assembled A (linear function) = 0 at interior nodes.  Exact on trilinear
    # elements for N >= 2: adj(J) has degree <= 2 per direction, so GLL
    # quadrature integrates grad v . adj(J) c exactly.
    N = 4
    m = _trilinear_box(3, 3, 3, N, seed=5)
    G, B, _ = geometry.factors(m)
    D = gll.derivative_matrix(N)
    glo, Pg = numbering.global_numbering(m)
    mask = numbering.dirichlet_mask(m, glo, Pg).reshape(B.shape)
    c = np.array([0.4, -1.3, 0.9])
    u = np.einsum("a,eakji->ekji", c, m.xyz)
    w = numbering.gs(operator.ax_local(u, G, B, D), glo, Pg)
    interior = mask > 0
    assert np.abs(w[interior]).max() < 1e-12 * np.abs(w).max()
    # the same with the transposed metric J^{-T} J^{-1} must fail
    J = geometry.jacobian(m)
    Jinv = np.linalg.inv(J)
    Mt = np.einsum("...ab,...ac->...bc", Jinv, Jinv)
    Gt = G.copy()
    for cidx, (p, q) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        Gt[:, cidx] = B * Mt[..., p, q]
    wt = numbering.gs(operator.ax_local(u, Gt, B, D), glo, Pg)
    assert np.abs(wt[interior]).max() > 1e-6 * np.abs(wt).max()
