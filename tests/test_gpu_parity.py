"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs (element by element), at sizes the oracle finishes in
seconds that still span several kernel tiles and a ragged tail."""

import numpy as np
import pytest

from oracle import gll, mesh as omesh, numbering, operator, solver
from sem_inputs import forcing, vectors

pytestmark = pytest.mark.gpu

AX_TOL = 1e-12       # FP64 Ax: relative L2 error bound
AX32_TOL = 2e-6      # FP32 Ax against the FP64 oracle (single-precision rounding)


def _oracle_mesh(desc):
    if desc["kind"] == "box":
        return omesh.box(desc["nx"], desc["ny"], desc["nz"], desc["N"], desc.get("lx", 1.0), desc.get("ly", 1.0),
                         desc.get("lz", 1.0))
    return omesh.pipe(desc["nc"], desc["nr"], desc["nzp"], desc["N"], R=desc.get("R", 1.0), L=desc.get("L", 8.0),
                      a=desc.get("a"), beta=desc.get("beta", 2.0), periodic=desc.get("periodic", True))


CASES = {
    "box4_n7": dict(kind="box", nx=4, ny=4, nz=4, N=7),                     # 64 elements
    "box_ragged_n7": dict(kind="box", nx=3, ny=2, nz=1, N=7, lx=1.5, ly=1.0, lz=0.5),  # 6 el: ragged tail
    "pipe_n3": dict(kind="pipe", nc=2, nr=1, nzp=3, N=3, L=3.0),
    "pipe_n5": dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0),
    "pipe_open_n4": dict(kind="pipe", nc=2, nr=2, nzp=3, N=4, L=2.0, periodic=False),
    "box_n1": dict(kind="box", nx=5, ny=3, nz=2, N=1),
    "box_n2": dict(kind="box", nx=3, ny=3, nz=3, N=2),
    "pipe_n9": dict(kind="pipe", nc=2, nr=1, nzp=3, N=9, L=3.0),
    "pipe_n11": dict(kind="pipe", nc=2, nr=1, nzp=3, N=11, L=3.0),
}

_cache = {}


def setup(name):
    import torch
    import paper_2109_03592_gb300 as sem
    if name not in _cache:
        desc = CASES[name]
        _cache[name] = (sem.Mesh(desc), solver.Problem(_oracle_mesh(desc)))
    return _cache[name]


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_matches_oracle(name):
    m, P = setup(name)
    assert m.E == P.mesh.E and m.n_global == P.Pg
    np.testing.assert_allclose(m.coords().cpu().numpy(), P.mesh.xyz, rtol=0, atol=2e-15 * max(1.0, np.abs(P.mesh.xyz).max()))
    assert np.array_equal(m.global_ids(), P.glo)
    G, B = m.geometry()
    assert relerr(G.cpu().numpy(), P.G) < 1e-13
    assert relerr(B.cpu().numpy(), P.B) < 1e-13
    mult, mask = m.weights()
    assert np.array_equal(mult.cpu().numpy(), P.mult.astype(np.float64))
    assert np.array_equal(mask.cpu().numpy(), P.mask)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.7, 3.5)])
def test_ax_fp64(name, h1, h2):
    import torch
    m, P = setup(name)
    u = vectors.local_field(11, m.E, m.n)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.ax(to_gpu(u), w, h1, h2)
    ref = operator.ax_local(u, P.G, P.B, P.D, h1, h2)
    assert relerr(w.cpu().numpy(), ref) < AX_TOL


@pytest.mark.parametrize("name", ["box4_n7", "pipe_n5", "pipe_n11", "box_ragged_n7"])
def test_ax_fp32(name):
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = setup(name)
    u = vectors.local_field(12, m.E, m.n, np.float32)
    w = torch.empty(m.shape, dtype=torch.float32, device="cuda")
    m.ax(to_gpu(u), w, 1.0, 0.5, prec=sem.FP32)
    ref = operator.ax_local(u.astype(np.float64), P.G, P.B, P.D, 1.0, 0.5)
    assert relerr(w.cpu().numpy().astype(np.float64), ref) < AX32_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_gs_bit_exact(name):
    import paper_2109_03592_gb300 as sem
    m, P = setup(name)
    for dt, prec in [(np.float64, sem.FP64), (np.float32, sem.FP32)]:
        v = vectors.local_field(13, m.E, m.n, dt)
        t = to_gpu(v)
        m.gs(t, apply_mask=False, prec=prec)
        ref = numbering.gs(v, P.glo, P.Pg)
        assert np.array_equal(t.cpu().numpy(), ref)
        t = to_gpu(v)
        m.gs(t, apply_mask=True, prec=prec)
        assert np.array_equal(t.cpu().numpy(), (P.mask.astype(dt) * ref).astype(dt))


@pytest.mark.parametrize("name", ["box4_n7", "pipe_n3", "pipe_open_n4", "pipe_n9"])
def test_rhs_apply_jacobi(name):
    import torch
    m, P = setup(name)
    f = forcing.evaluate(P.mesh.xyz, forcing.random_modes(5, L=3.0))
    b = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.rhs(to_gpu(f), b)
    assert relerr(b.cpu().numpy(), P.rhs(f)) < 1e-13
    x = P.mask * vectors.local_field(14, m.E, m.n)
    x = numbering.gs(x, P.glo, P.Pg) / P.mult  # a continuous field
    y = torch.empty_like(b)
    m.apply(to_gpu(x), y, P.h1, P.h2)
    assert relerr(y.cpu().numpy(), P.A(x)) < AX_TOL
    mi = torch.empty_like(b)
    m.jacobi(mi, 1.0, 0.0)
    assert relerr(mi.cpu().numpy(), P.jacobi_inverse()) < 1e-13


def _residual(P, b, x):
    r = b - P.A(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


@pytest.mark.parametrize("name", ["box4_n7", "pipe_n5", "pipe_open_n4", "box_n2"])
def test_pcg_fp64_matches_oracle(name):
    import torch
    m, P = setup(name)
    f = forcing.evaluate(P.mesh.xyz, forcing.random_modes(6, L=3.0))
    b = P.rhs(f)
    ref = solver.pcg(P, b, tol=1e-10)
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), x, tol=1e-10)
    assert res["status"] == 0
    assert abs(res["iters"] - ref.iters) <= 2, (res, ref.iters)
    xs = x.cpu().numpy()
    assert _residual(P, b, xs) <= 1.1e-10
    assert np.sqrt(P.dot(xs - ref.x, xs - ref.x) / P.dot(ref.x, ref.x)) < 1e-8


def test_pcg_helmholtz_and_mixed():
    import torch
    import paper_2109_03592_gb300 as sem
    m, _ = setup("pipe_n5")
    P = solver.Problem(_oracle_mesh(CASES["pipe_n5"]), 1.0, 2.0)
    f = forcing.evaluate(P.mesh.xyz, forcing.random_modes(8, L=2.0))
    b = P.rhs(f)
    ref = solver.pcg(P, b, tol=1e-12)
    for prec in (sem.FP64, sem.MIXED):
        x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
        res = m.solve(to_gpu(b), x, tol=1e-10, h1=1.0, h2=2.0, prec=prec)
        assert res["status"] == 0, res
        xs = x.cpu().numpy()
        assert _residual(P, b, xs) <= (1.1e-10 if prec == sem.FP64 else 1e-10)
        err = np.sqrt(P.dot(xs - ref.x, xs - ref.x) / P.dot(ref.x, ref.x))
        assert err < 1e-8, err
        if prec == sem.MIXED:
            assert res["outer_iters"] >= 2


def test_manufactured_solution_box():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = setup("box4_n7")
    f = forcing.manufactured(P.mesh.xyz)
    bt = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.rhs(to_gpu(f), bt)
    ustar = forcing.manufactured_solution(P.mesh.xyz)
    for prec in (sem.FP64, sem.MIXED):
        x = torch.zeros_like(bt)
        res = m.solve(bt, x, tol=1e-10, prec=prec)
        assert res["status"] == 0
        assert np.abs(x.cpu().numpy() - ustar).max() < 1e-9


def test_zero_rhs_and_initial_guess():
    import torch
    m, P = setup("box4_n7")
    b = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    x = torch.ones_like(b)
    res = m.solve(b, x)
    assert res["iters"] == 0 and res["status"] == 0 and float(x.abs().max()) == 0.0
    bn = P.rhs(forcing.manufactured(P.mesh.xyz))
    exact = solver.pcg(P, bn, tol=1e-13).x
    x = to_gpu(exact)
    res = m.solve(to_gpu(bn), x, tol=1e-10)
    assert res["iters"] == 0


@pytest.mark.parametrize("N", [1, 2, 7])
def test_single_element_degenerate_systems(N):
    """One element with Dirichlet faces all round: at N = 1 every node lies on
    the boundary (no unknowns: b = 0 and both solves return x = 0 at once);
    at N = 2 one free node (Jacobi-PCG is exact in one step); at N = 7 a 6^3
    interior, on one ragged tile of the element-blocked kernels.  Ax, QQ^T
    and the FP64 and mixed solves against the oracle."""
    import torch
    import paper_2109_03592_gb300 as sem
    desc = dict(kind="box", nx=1, ny=1, nz=1, N=N, lx=0.7, ly=1.0, lz=1.3)
    m = sem.Mesh(desc)
    P = solver.Problem(_oracle_mesh(desc))
    assert m.E == 1 and m.n_global == P.Pg
    u = vectors.local_field(5, 1, N + 1)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.ax(to_gpu(u), w, 1.0, 0.0)
    assert relerr(w.cpu().numpy(), operator.ax_local(u, P.G, P.B, P.D)) < AX_TOL
    m.gs(w, apply_mask=True)
    ref = P.mask * P.gs(operator.ax_local(u, P.G, P.B, P.D))
    np.testing.assert_allclose(w.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(3, L=1.3)))
    for prec in (sem.FP64, sem.MIXED):
        x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
        res = m.solve(to_gpu(b), x, tol=1e-10, prec=prec)
        assert res["status"] == 0, res
        xs = x.cpu().numpy()
        if N == 1:
            assert not b.any() and res["iters"] == 0 and not xs.any()
            continue
        assert _residual(P, b, xs) <= 1.1e-10
        if N == 2 and prec == sem.FP64:  # the mixed solve adds FP64 residual replacements
            assert res["iters"] == 1


def test_determinism():
    import torch
    m, P = setup("pipe_n5")
    u = to_gpu(vectors.local_field(21, m.E, m.n))
    w1 = torch.empty_like(u)
    w2 = torch.empty_like(u)
    m.ax(u, w1)
    m.ax(u, w2)
    assert torch.equal(w1, w2)
    b = to_gpu(P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(2, L=2.0))))
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    r1 = m.solve(b, x1)
    r2 = m.solve(b, x2)
    assert r1["iters"] == r2["iters"] and torch.equal(x1, x2)


def test_inverted_element_rejected():
    import paper_2109_03592_gb300 as sem
    om = omesh.box(2, 1, 1, 3)
    xyz = om.xyz.copy()
    xyz[1, 0] = xyz[1, 0, :, :, ::-1]  # mirror element 1 in x: det J < 0
    vert = sem.mesh_vertices(dict(kind="box", nx=2, ny=1, nz=1, N=3))
    desc = dict(kind="explicit", N=3, xyz=xyz, vert=vert, dirichlet_face=om.dirichlet_face.astype(np.uint8))
    with pytest.raises(sem.SemError) as ei:
        sem.Mesh(desc)
    assert ei.value.status == sem.SEM_ERR_BAD_MESH


def test_explicit_mesh_equals_generator():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = setup("pipe_n3")
    vert = sem.mesh_vertices(CASES["pipe_n3"])
    desc = dict(kind="explicit", N=3, xyz=P.mesh.xyz, vert=vert, dirichlet_face=P.mesh.dirichlet_face.astype(np.uint8))
    me = sem.Mesh(desc)
    assert np.array_equal(me.global_ids(), P.glo)
    u = to_gpu(vectors.local_field(3, m.E, m.n))
    w = torch.empty_like(u)
    me.ax(u, w)
    assert relerr(w.cpu().numpy(), operator.ax_local(u.cpu().numpy(), P.G, P.B, P.D)) < AX_TOL


@pytest.mark.parametrize("kernel", ["native", "df"])
@pytest.mark.parametrize("name", ["box_ragged_n7", "pipe_n5", "pipe_n11", "box_n1"])
def test_ax_fp64_both_kernels(kernel, name, monkeypatch):
    """Both FP64 local-operator kernels (native FP64 and double-float) meet
    the FP64 bound, whichever the autotuner picks."""
    import torch
    import paper_2109_03592_gb300 as sem
    monkeypatch.setenv("SEM_FP64_KERNEL", kernel)
    m = sem.Mesh(CASES[name])
    assert m.fp64_double_float() == (kernel == "df")
    _, P = setup(name)
    u = vectors.local_field(31, m.E, m.n)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    for h1, h2 in [(1.0, 0.0), (0.3, 7.0)]:
        m.ax(to_gpu(u), w, h1, h2)
        ref = operator.ax_local(u, P.G, P.B, P.D, h1, h2)
        assert relerr(w.cpu().numpy(), ref) < AX_TOL
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(4, L=3.0)))
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), x, tol=1e-10)
    assert res["status"] == 0 and _residual(P, b, x.cpu().numpy()) <= 1.1e-10


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("name,h2", [("pipe_n5", 0.0), ("box4_n7", 0.0), ("pipe_open_n4", 1.5)])
def test_mixed_variants_match_oracle(refine, name, h2):
    """Reliable updates (refine=0, the default) and restarted refinement
    (refine=1) against the oracle's versions of the same algorithms."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, _ = setup(name)
    P = solver.Problem(_oracle_mesh(CASES[name]), 1.0, h2)
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(12, L=2.0)))
    if refine == 0:
        ref = solver.pcg_mixed_reliable(P, b, tol=1e-10)
    else:
        ref = solver.pcg_mixed(P, b, tol=1e-10, inner_tol=1e-4)
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), x, tol=1e-10, h1=1.0, h2=h2, prec=sem.MIXED, refine=refine, inner_tol=1e-4)
    assert res["status"] == 0, res
    assert _residual(P, b, x.cpu().numpy()) <= 1e-10
    # FP32 rounding differs between numpy and the GPU: counts agree to ~10%
    assert abs(res["iters"] - ref.iters) <= 0.1 * ref.iters + 3, (res, ref.iters)
    fp64 = solver.pcg(P, b, tol=1e-10)
    if refine == 0:
        assert res["iters"] <= 1.3 * fp64.iters + 5


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["box_ragged_n7", "pipe_n5", "pipe_n11", "box4_n7", "box_n1"])
def test_fp32_variants(variant, name, monkeypatch):
    """Every FP32 local-operator variant (register kernels 0/1, bulk-copy
    pipelined kernels 2/3 for even n) against the oracle, plain and inside
    the fused CG iteration (mixed-precision solve)."""
    import torch
    import paper_2109_03592_gb300 as sem
    monkeypatch.setenv("SEM_FP32_VARIANT", str(variant))
    m = sem.Mesh(CASES[name])
    if m.ax_variant(sem.FP32) != variant:
        assert variant >= 2 and m.n % 2 == 1  # bulk-copy kernels exist for even n only
        pytest.skip("variant not available for odd n")
    _, P = setup(name)
    u = vectors.local_field(41, m.E, m.n, np.float32)
    w = torch.empty(m.shape, dtype=torch.float32, device="cuda")
    for h1, h2 in [(1.0, 0.0), (0.4, 3.0)]:
        m.ax(to_gpu(u), w, h1, h2, prec=sem.FP32)
        m.check()
        ref = operator.ax_local(u.astype(np.float64), P.G, P.B, P.D, h1, h2)
        assert relerr(w.cpu().numpy().astype(np.float64), ref) < AX32_TOL
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(4, L=3.0)))
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), x, tol=1e-10, prec=sem.MIXED)
    assert res["status"] == 0 and _residual(P, b, x.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["box_ragged_n7", "box4_n7", "pipe_n3", "pipe_n5", "pipe_n9", "pipe_n11", "box_n1",
                                  "pipe_open_n4"])
def test_fp64_double_float_variants(variant, name, monkeypatch):
    """Every double-float FP64 local-operator variant (direct kernels 0/1,
    even-odd kernels 2/3 for even n) meets the FP64 bound, plain (h1 = 1 uses
    the pre-split coefficient table, h1 != 1 the FP64 one) and inside the
    fused CG iteration of the FP64 solve."""
    import torch
    import paper_2109_03592_gb300 as sem
    monkeypatch.setenv("SEM_FP64_DF_VARIANT", str(variant))
    m = sem.Mesh(CASES[name])
    if m.ax_variant(sem.FP64) != variant:
        assert variant >= 2 and m.n % 2 == 1  # even-odd kernels exist for even n only
        pytest.skip("variant not available for odd n")
    assert m.fp64_double_float()
    _, P = setup(name)
    u = vectors.local_field(43, m.E, m.n)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    for h1, h2 in [(1.0, 0.0), (0.3, 7.0), (2.5, 0.0), (1.0, 1e-2)]:
        m.ax(to_gpu(u), w, h1, h2)
        ref = operator.ax_local(u, P.G, P.B, P.D, h1, h2)
        assert relerr(w.cpu().numpy(), ref) < AX_TOL, (h1, h2)
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(4, L=3.0)))
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), x, tol=1e-10)
    assert res["status"] == 0 and _residual(P, b, x.cpu().numpy()) <= 1.1e-10
    ref = solver.pcg(P, b, tol=1e-10)
    assert abs(res["iters"] - ref.iters) <= 2


@pytest.mark.parametrize("kernel", ["native", "df0", "df1", "df2", "df3"])
@pytest.mark.parametrize("name", ["box4_n7", "pipe_n5", "pipe_n11", "box_ragged_n7"])
def test_ax_fp64_smooth_fields(kernel, name, monkeypatch):
    """A smooth field with a mean: the stiffness part cancels the mean, so
    rounding of its low-order bits is amplified; every FP64 kernel must still
    meet the FP64 bound (the double-float kernels shift by the element's first
    value before contracting).  A mean of 2 costs FP64 arithmetic itself ~1e-13
    here; much larger means are not a 1e-12 test of anything, because the
    oracle's rounded D no longer annihilates constants to that level."""
    import torch
    import paper_2109_03592_gb300 as sem
    if kernel == "native":
        monkeypatch.setenv("SEM_FP64_KERNEL", "native")
    else:
        monkeypatch.setenv("SEM_FP64_DF_VARIANT", kernel[2])
    m = sem.Mesh(CASES[name])
    if kernel != "native" and m.ax_variant(sem.FP64) != int(kernel[2]):
        pytest.skip("variant not available for odd n")
    assert m.fp64_double_float() == (kernel != "native")
    _, P = setup(name)
    x, y, z = (P.mesh.xyz[:, a] for a in range(3))
    for off in (0.0, 2.0):
        u = np.sin(np.pi * x) * np.cos(0.5 * np.pi * y) * np.sin(0.7 * z + 0.3) + off
        w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
        for h1, h2 in [(1.0, 0.0), (0.3, 7.0)]:
            m.ax(to_gpu(u), w, h1, h2)
            ref = operator.ax_local(u, P.G, P.B, P.D, h1, h2)
            assert relerr(w.cpu().numpy(), ref) < AX_TOL, (off, h1, h2, relerr(w.cpu().numpy(), ref))


def test_fp32_bulk_copy_kernel_unaligned_input():
    """A caller's u that is not 16-byte aligned falls back to a register kernel."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = setup("box4_n7")
    u = vectors.local_field(43, m.E, m.n, np.float32)
    buf = torch.zeros(u.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = to_gpu(u).reshape(-1)
    uu = buf[1:]
    assert uu.data_ptr() % 16 != 0
    w = torch.empty(u.size, dtype=torch.float32, device="cuda")
    m.ax(uu, w, 1.0, 0.0, prec=sem.FP32)
    m.check()
    ref = operator.ax_local(u.astype(np.float64), P.G, P.B, P.D)
    assert relerr(w.cpu().numpy().reshape(u.shape).astype(np.float64), ref) < AX32_TOL
