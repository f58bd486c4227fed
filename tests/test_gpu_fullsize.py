"""Parity at full size: the benchmark's O-grid pipe (E = 262,144, N = 7, the
configuration bench.py times) and the large cases (E = 131,072 at N = 11;
E = 1,048,576 at N = 7, ~3.6e8 global nodes).  Outputs the oracle can compute
one element at a time are compared on sampled elements; the rest through
properties that hold at any size."""

import numpy as np
import pytest

from oracle import geometry, gll, mesh as omesh, operator
from sem_inputs import configs, forcing

pytestmark = pytest.mark.gpu

BENCH = "pipe262144_n7"
SAMPLE = 48


@pytest.fixture(scope="module", params=[BENCH, "pipe131072_n11", "pipe1048576_n7"])
def big(request):
    import torch
    import paper_2109_03592_gb300 as sem
    desc = configs.mesh_desc(request.param)
    m = sem.Mesh(desc)
    rng = np.random.default_rng(7)
    els = np.sort(rng.choice(m.E, SAMPLE, replace=False))
    om = omesh.pipe(desc["nc"], desc["nr"], desc["nzp"], desc["N"], R=desc["R"], L=desc["L"], a=desc["a"],
                    beta=desc["beta"], periodic=True, elements=els)
    G, B, _ = geometry.factors(om)
    D = gll.derivative_matrix(desc["N"])
    yield m, desc, els, om, G, B, D
    m.close()
    del m
    import gc
    gc.collect()
    torch.cuda.empty_cache()


def _rows(t, els):
    import torch
    return t[torch.as_tensor(els, device=t.device)].cpu().numpy()


def test_numbering_properties(big):
    m, desc, els, om, G, B, D = big
    assert m.n_global == omesh.pipe_global_node_count(desc["nc"], desc["nr"], desc["nzp"], desc["N"])
    glo = m.global_ids()
    assert glo[0] == 0 and np.all(np.diff(np.maximum.accumulate(glo)) <= 1)  # first touch
    mult = np.bincount(glo)
    assert mult.size == m.n_global and mult.min() >= 1 and mult.max() == 8
    hist = np.bincount(mult)
    # 3: z-edges through the O-grid square corners (3 elements in the plane); 6: their vertices
    assert hist[6] > 0 and hist[3] > 0 and set(np.nonzero(hist)[0]) <= {1, 2, 3, 4, 6, 8}
    del mult, hist
    # sampled elements: the library's ids, relabelled in first-touch order over
    # the sample, equal the oracle's coordinate-based numbering of the sample
    from oracle import numbering
    n3 = m.n ** 3
    ids = np.concatenate([glo[e * n3:(e + 1) * n3] for e in els])
    _, first = np.unique(ids, return_index=True)
    rank = np.empty(first.size, dtype=np.int64)
    rank[np.argsort(first)] = np.arange(first.size)
    relabel = rank[np.searchsorted(np.unique(ids), ids)]
    og, opg = numbering.global_numbering(om)
    assert np.array_equal(relabel, og)


def test_coords_geometry_sampled(big):
    m, desc, els, om, G, B, D = big
    import torch
    xyz = m.coords()
    np.testing.assert_allclose(_rows(xyz, els), om.xyz, rtol=0, atol=4e-15)
    del xyz
    Gd, Bd = m.geometry()
    g = _rows(Gd, els)
    # elements of aspect ratio ~15 (0.0156 long in z) amplify the rounding of
    # J (FMA dot products here, einsum in the oracle) through J^-1 J^-T; the
    # binding bar is Ax <= 1e-12 below
    assert np.linalg.norm(g - G) / np.linalg.norm(G) < 5e-13
    assert np.linalg.norm(_rows(Bd, els) - B) / np.linalg.norm(B) < 5e-13
    del Gd, Bd
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_ax_sampled(big, prec, tol):
    import torch
    import paper_2109_03592_gb300 as sem
    m, desc, els, om, G, B, D = big
    gen = torch.Generator(device="cuda").manual_seed(11)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.randn(m.shape, dtype=torch.float64, device="cuda", generator=gen).to(dt)
    w = torch.empty_like(u)
    for h1, h2 in [(1.0, 0.0), (0.5, 2.0)]:
        m.ax(u, w, h1, h2, prec=sem.FP64 if prec == "fp64" else sem.FP32)
        m.check()
        us = _rows(u, els).astype(np.float64)
        ref = operator.ax_local(us, G, B, D, h1, h2)
        got = _rows(w, els).astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol


def test_gs_properties_full_size(big):
    import torch
    import paper_2109_03592_gb300 as sem
    m, desc, els, om, G, B, D = big
    mult, mask = m.weights()
    v = 1.0 / mult
    m.gs(v, apply_mask=False)
    assert float((v - 1.0).abs().max()) <= 4e-16
    del v
    # random field: every copy of a node holds the ascending-index sum of the copies
    glo = m.global_ids()
    gen = torch.Generator(device="cuda").manual_seed(3)
    r = torch.randn(m.shape, dtype=torch.float32, device="cuda", generator=gen)
    before = r.reshape(-1).cpu().numpy()
    m.gs(r, apply_mask=True, prec=sem.FP32)
    after = r.reshape(-1).cpu().numpy()
    maskh = mask.reshape(-1).cpu().numpy()
    rng = np.random.default_rng(5)
    for l0 in rng.choice(m.n_local, 40, replace=False):
        copies = np.nonzero(glo == glo[l0])[0]
        s = before[copies[0]]
        for c in copies[1:]:
            s = np.float32(s + before[c])
        expect = s if maskh[l0] > 0 else np.float32(0.0)
        assert np.all(after[copies] == expect)


@pytest.mark.parametrize("prec_name", ["MIXED", "FP64"])
def test_solve_sampled_residual(big, prec_name):
    """The bench's solve (mixed precision, reliable updates) and the plain
    FP64 PCG, tol 1e-10, on every full-size mesh (E = 262,144 and 1,048,576
    at N = 7; E = 131,072 at N = 11): the residual at element-interior points
    of sampled elements, recomputed by the oracle from x, is bounded by
    ||r|| <= 1e-10 ||b|| (an interior point has one copy, so |r_l| <= ||r||)."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, desc, els, om, G, B, D = big
    xyz = m.coords()
    modes = forcing.random_modes(2, L=desc["L"])
    f = forcing.evaluate_torch(xyz, modes)
    del xyz
    b = torch.empty_like(f)
    m.rhs(f, b)
    mult, mask = m.weights()
    bnorm = float(torch.sqrt((b * b / mult).sum()))
    del mult, mask
    x = torch.zeros_like(b)
    res = m.solve(b, x, tol=1e-10, prec=getattr(sem, prec_name))
    assert res["status"] == 0 and res["rel_res"] <= 1e-10
    xs = _rows(x, els)
    fs = forcing.evaluate(om.xyz, modes)
    Ax = operator.ax_local(xs, G, B, D)
    r = B * fs - Ax  # element-interior points: no assembly, no mask
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(r[inner]).max() <= 1.05e-10 * bnorm
    del f, b, x
    torch.cuda.empty_cache()
