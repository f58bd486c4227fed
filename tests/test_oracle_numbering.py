"""Pins for global numbering and QQ^T (Sec. 2, exchange of element face values)."""

import numpy as np
import pytest

from oracle import mesh, numbering


def _brute_numbering(m, tol=1e-9):
    """O(P^2) first-touch numbering by pairwise distances (tiny meshes)."""
    pts = numbering.local_points(m).copy()
    if m.period is not None:
        pts[pts[:, 2] >= m.period - tol, 2] -= m.period
    P = len(pts)
    glo = -np.ones(P, dtype=np.int64)
    nxt = 0
    for l in range(P):
        if glo[l] >= 0:
            continue
        same = np.where(np.abs(pts - pts[l]).max(axis=1) < tol)[0]
        glo[same] = nxt
        nxt += 1
    return glo, nxt


@pytest.mark.parametrize("maker", [
    lambda: mesh.box(2, 1, 2, 2),
    lambda: mesh.pipe(2, 1, 2, 2, L=2.0),
    lambda: mesh.pipe(2, 1, 2, 2, L=2.0, periodic=False),
])
def test_kdtree_numbering_equals_brute_force(maker):
    m = maker()
    g1, p1 = numbering.global_numbering(m)
    g2, p2 = _brute_numbering(m)
    assert p1 == p2
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("nx,ny,nz,N", [(4, 4, 4, 3), (2, 3, 1, 5), (1, 1, 1, 2)])
def test_box_counts(nx, ny, nz, N):
    m = mesh.box(nx, ny, nz, N)
    glo, Pg = numbering.global_numbering(m)
    assert Pg == mesh.box_global_node_count(nx, ny, nz, N)
    mult = numbering.multiplicity(glo, Pg)
    assert abs(np.sum(1.0 / mult) - Pg) < 1e-9
    assert mult.max() == min(8, 2 ** ((nx > 1) + (ny > 1) + (nz > 1)))
    # first-touch: ids appear in increasing order of first occurrence
    seen = np.maximum.accumulate(glo)
    assert glo[0] == 0 and np.all(glo <= np.concatenate([[0], seen[:-1] + 1]))


@pytest.mark.parametrize("nc,nr,nzp,N,periodic", [(2, 1, 2, 3, True), (4, 2, 3, 2, True), (2, 2, 2, 2, False)])
def test_pipe_counts_and_multiplicities(nc, nr, nzp, N, periodic):
    m = mesh.pipe(nc, nr, nzp, N, L=3.0, periodic=periodic)
    glo, Pg = numbering.global_numbering(m)
    assert Pg == mesh.pipe_global_node_count(nc, nr, nzp, N, periodic)
    mult = numbering.multiplicity(glo, Pg)
    assert mult.max() == 8
    # the four O-grid square corners are shared by 3 elements in the plane
    hist = np.bincount(np.bincount(glo))
    assert hist[6] > 0
    # histogram check against a direct coordinate count
    pts = numbering.local_points(m).copy()
    if m.period is not None:
        pts[pts[:, 2] >= m.period - 1e-9, 2] -= m.period
    key = np.round(pts * 1e7).astype(np.int64)
    _, counts = np.unique(key, axis=0, return_counts=True)
    assert np.array_equal(np.bincount(counts, minlength=hist.size), hist)


def test_gs_pins():
    m = mesh.pipe(2, 1, 2, 3, L=2.0)
    glo, Pg = numbering.global_numbering(m)
    mult = numbering.multiplicity(glo, Pg)
    np.testing.assert_allclose(numbering.gs(1.0 / mult, glo, Pg), np.ones(glo.size), rtol=0, atol=4e-16)
    # indicator of one copy spreads to every copy of its node
    l0 = int(np.argmax(mult))
    v = np.zeros(glo.size)
    v[l0] = 1.0
    s = numbering.gs(v, glo, Pg)
    assert np.array_equal(s == 1.0, glo == glo[l0]) and s.sum() == mult[l0]
    # np.add.at order == plain left-to-right loop, bit for bit, in fp64 and fp32
    rng = np.random.default_rng(3)
    for dt in (np.float64, np.float32):
        v = rng.standard_normal(glo.size).astype(dt)
        assert np.array_equal(numbering.gs(v, glo, Pg), numbering.gs_loop(v, glo, Pg))


def test_dirichlet_mask_pipe():
    m = mesh.pipe(2, 1, 2, 3, L=2.0)
    glo, Pg = numbering.global_numbering(m)
    mask = numbering.dirichlet_mask(m, glo, Pg)
    pts = numbering.local_points(m)
    r = np.hypot(pts[:, 0], pts[:, 1])
    assert np.array_equal(mask == 0.0, np.abs(r - 1.0) < 1e-12)
