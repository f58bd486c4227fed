"""GPU parity for per-point coefficients h1(i,j,k,e), h2(i,j,k,e)
(sem_mesh_set_coefficients; Alg. 1 reads h1 per local point) against the
oracle's per-point operator, on every local-operator kernel, in the solvers,
the batch engine and a projection space."""

import numpy as np
import pytest

from oracle import mesh as omesh, operator, projection, solver
from sem_inputs import coefficients, forcing, vectors

pytestmark = pytest.mark.gpu

AX_TOL = 1e-12
AX32_TOL = 2e-6

CASES = {
    "box_ragged_n7": dict(kind="box", nx=3, ny=2, nz=1, N=7, lx=1.5, ly=1.0, lz=0.5),
    "pipe_n5": dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0),
    "pipe_n11": dict(kind="pipe", nc=2, nr=1, nzp=3, N=11, L=3.0),
    "pipe_open_n4": dict(kind="pipe", nc=2, nr=2, nzp=3, N=4, L=2.0, periodic=False),
    "box_n1": dict(kind="box", nx=5, ny=3, nz=2, N=1),
}


def _om(d):
    if d["kind"] == "box":
        return omesh.box(d["nx"], d["ny"], d["nz"], d["N"], d.get("lx", 1.0), d.get("ly", 1.0), d.get("lz", 1.0))
    return omesh.pipe(d["nc"], d["nr"], d["nzp"], d["N"], L=d["L"], periodic=d.get("periodic", True))


def _fields(om, seed=21):
    return coefficients.viscosity(seed, om.xyz), coefficients.mass_coefficient(seed + 1, om.xyz)


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _residual(P, b, x):
    r = b - P.A(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


def _mesh(name, monkeypatch, kernel):
    import paper_2109_03592_gb300 as sem
    if kernel == "native":
        monkeypatch.setenv("SEM_FP64_KERNEL", "native")
    else:
        monkeypatch.setenv("SEM_FP64_KERNEL", "df")
        monkeypatch.setenv("SEM_FP64_DF_VARIANT", kernel[2:])
    return sem.Mesh(CASES[name])


@pytest.mark.parametrize("kernel", ["native", "df0", "df1", "df2", "df3"])
@pytest.mark.parametrize("name", list(CASES))
def test_ax_per_point(kernel, name, monkeypatch):
    import torch
    import paper_2109_03592_gb300 as sem
    m = _mesh(name, monkeypatch, kernel)
    if kernel != "native" and m.ax_variant(sem.FP64) != int(kernel[2:]):
        pytest.skip("even-odd kernels exist for even n only")
    om = _om(CASES[name])
    P = solver.Problem(om)
    h1, h2 = _fields(om)
    m.set_coefficients(to_gpu(h1), to_gpu(h2))
    u = vectors.local_field(51, m.E, m.n)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    for s1, s2 in [(1.0, 0.0), (0.5, 2.0), (1.0, 1.0)]:
        m.ax(to_gpu(u), w, s1, s2)
        ref = operator.ax_local(u, P.G, P.B, P.D, s1 * h1, s2 * h2)
        assert relerr(w.cpu().numpy(), ref) < AX_TOL, (s1, s2)
    u32 = u.astype(np.float32)
    w32 = torch.empty(m.shape, dtype=torch.float32, device="cuda")
    m.ax(to_gpu(u32), w32, 1.0, 1.0, prec=sem.FP32)
    m.check()
    ref = operator.ax_local(u32.astype(np.float64), P.G, P.B, P.D, h1, h2)
    assert relerr(w32.cpu().numpy().astype(np.float64), ref) < AX32_TOL


@pytest.mark.parametrize("name", ["box_ragged_n7", "pipe_n5", "pipe_open_n4"])
def test_apply_jacobi_and_solves(name):
    import torch
    import paper_2109_03592_gb300 as sem
    m = sem.Mesh(CASES[name])
    om = _om(CASES[name])
    h1, h2 = _fields(om)
    m.set_coefficients(to_gpu(h1), to_gpu(h2))
    P = solver.Problem(om, h1, h2)
    x = vectors.local_field(52, m.E, m.n)
    from oracle import numbering
    x = numbering.gs(P.mask * x, P.glo, P.Pg) / P.mult  # continuous
    y = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.apply(to_gpu(x), y, 1.0, 1.0)
    assert relerr(y.cpu().numpy(), P.A(x)) < AX_TOL
    mi = torch.empty_like(y)
    m.jacobi(mi, 1.0, 1.0)
    assert relerr(mi.cpu().numpy(), P.jacobi_inverse()) < 1e-13
    b = P.rhs(forcing.evaluate(om.xyz, forcing.random_modes(53, L=2.0)))
    ref = solver.pcg(P, b, tol=1e-10)
    for prec in (sem.FP64, sem.MIXED):
        xg = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
        res = m.solve(to_gpu(b), xg, tol=1e-10, h1=1.0, h2=1.0, prec=prec)
        assert res["status"] == 0, res
        xs = xg.cpu().numpy()
        assert _residual(P, b, xs) <= (1.1e-10 if prec == sem.FP64 else 1e-10)
        assert np.sqrt(P.dot(xs - ref.x, xs - ref.x) / P.dot(ref.x, ref.x)) < 1e-8
        if prec == sem.FP64:
            assert abs(res["iters"] - ref.iters) <= 2, (res, ref.iters)


def test_coefficient_change_between_solves():
    """The solver's cached workspace (Jacobi inverse, captured iteration
    graphs) follows a change of coefficients between solves with the same
    scalar h1, h2."""
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["pipe_n5"]
    m = sem.Mesh(d)
    om = _om(d)
    f = forcing.evaluate(om.xyz, forcing.random_modes(59, L=2.0))
    problems = [solver.Problem(om, 1.0, 1.0)]
    for seed in (81, 83):
        h1, h2 = _fields(om, seed)
        problems.append((solver.Problem(om, h1, h2), h1, h2))
    for prec in (sem.FP64, sem.MIXED):
        for k, item in enumerate(problems):
            if k == 0:
                P = item
                m.set_coefficients(None, None)
            else:
                P, h1, h2 = item
                m.set_coefficients(to_gpu(h1), to_gpu(h2))
            b = P.rhs(f)
            x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
            res = m.solve(to_gpu(b), x, tol=1e-10, h1=1.0, h2=1.0, prec=prec)
            assert res["status"] == 0, (prec, k, res)
            assert _residual(P, b, x.cpu().numpy()) <= (1.1e-10 if prec == sem.FP64 else 1e-10)


def test_stiffness_only_coefficient_and_poisson():
    """h1 per point with h2 left constant, solved as a Poisson problem
    (h2 = 0): the h1 copies alone."""
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["pipe_n5"]
    m = sem.Mesh(d)
    om = _om(d)
    h1, _ = _fields(om, 31)
    m.set_coefficients(to_gpu(h1), None)
    P = solver.Problem(om, h1, 0.0)
    b = P.rhs(forcing.evaluate(om.xyz, forcing.random_modes(54, L=2.0)))
    xg = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = m.solve(to_gpu(b), xg, tol=1e-10, prec=sem.MIXED)
    assert res["status"] == 0 and _residual(P, b, xg.cpu().numpy()) <= 1e-10
    # and a constant h2 = 3 on top of it
    P3 = solver.Problem(om, h1, 3.0)
    u = vectors.local_field(55, m.E, m.n)
    w = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    m.ax(to_gpu(u), w, 1.0, 3.0)
    assert relerr(w.cpu().numpy(), operator.ax_local(u, P3.G, P3.B, P3.D, h1, 3.0)) < AX_TOL


def test_reset_restores_the_plain_operator_bit_for_bit():
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["box_ragged_n7"]
    m = sem.Mesh(d)
    om = _om(d)
    u = to_gpu(vectors.local_field(56, m.E, m.n))
    w0, w1 = (torch.empty(m.shape, dtype=torch.float64, device="cuda") for _ in range(2))
    j0, j1 = torch.empty_like(w0), torch.empty_like(w0)
    m.ax(u, w0, 0.7, 2.0)
    m.jacobi(j0, 0.7, 2.0)
    h1, h2 = _fields(om)
    m.set_coefficients(to_gpu(h1), to_gpu(h2))
    m.ax(u, w1, 0.7, 2.0)
    assert not torch.equal(w0, w1)
    m.set_coefficients(None, None)
    m.ax(u, w1, 0.7, 2.0)
    m.jacobi(j1, 0.7, 2.0)
    assert torch.equal(w0, w1) and torch.equal(j0, j1)


def test_constant_arrays_equal_scalars():
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["pipe_n5"]
    m = sem.Mesh(d)
    u = to_gpu(vectors.local_field(57, m.E, m.n))
    w0, w1 = (torch.empty(m.shape, dtype=torch.float64, device="cuda") for _ in range(2))
    m.ax(u, w0, 0.7, 3.0)
    m.set_coefficients(torch.full(m.shape, 0.7, dtype=torch.float64, device="cuda"),
                       torch.full(m.shape, 3.0, dtype=torch.float64, device="cuda"))
    m.ax(u, w1, 1.0, 1.0)
    assert relerr(w1.cpu().numpy(), w0.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("bad", ["h1_zero", "h1_negative", "h1_nan", "h1_inf", "h2_negative", "h2_nan"])
def test_invalid_coefficients_rejected_and_mesh_unchanged(bad):
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["pipe_n5"]
    m = sem.Mesh(d)
    om = _om(d)
    h1, h2 = _fields(om)
    m.set_coefficients(to_gpu(h1), to_gpu(h2))
    u = to_gpu(vectors.local_field(58, m.E, m.n))
    w0, w1 = (torch.empty(m.shape, dtype=torch.float64, device="cuda") for _ in range(2))
    m.ax(u, w0, 1.0, 1.0)
    b1, b2 = h1.copy(), h2.copy()
    target, value = {"h1_zero": (b1, 0.0), "h1_negative": (b1, -1.0), "h1_nan": (b1, np.nan),
                     "h1_inf": (b1, np.inf), "h2_negative": (b2, -0.5), "h2_nan": (b2, np.nan)}[bad]
    target.reshape(-1)[target.size // 3] = value
    with pytest.raises(sem.SemError):
        m.set_coefficients(to_gpu(b1), to_gpu(b2))
    m.ax(u, w1, 1.0, 1.0)
    assert torch.equal(w0, w1)
    with pytest.raises(ValueError):
        m.set_coefficients(torch.ones(m.n_local - 1, dtype=torch.float64, device="cuda"), None)


def test_batch_with_per_point_coefficients():
    """Requests on meshes with and without per-point coefficients in one
    batch: each equals its batch of one and meets the oracle's residual."""
    import torch
    import paper_2109_03592_gb300 as sem
    descs = [dict(kind="pipe", nc=2, nr=1, nzp=3, N=5, L=3.0), dict(kind="box", nx=3, ny=3, nz=3, N=5)]
    meshes, probs, bs = [], [], []
    for i, d in enumerate(descs):
        om = omesh.pipe(d["nc"], d["nr"], d["nzp"], d["N"], L=d["L"]) if d["kind"] == "pipe" else \
            omesh.box(d["nx"], d["ny"], d["nz"], d["N"])
        m = sem.Mesh(d)
        if i == 0:
            h1, h2 = _fields(om, 61)
            m.set_coefficients(to_gpu(h1), to_gpu(h2))
            P = solver.Problem(om, h1, h2)
        else:
            P = solver.Problem(om, 1.0, 1.0)
        meshes.append(m)
        probs.append(P)
        bs.append(to_gpu(P.rhs(forcing.evaluate(om.xyz, forcing.random_modes(62 + i, L=3.0)))))

    def run(idx):
        xs = [torch.zeros_like(bs[i]) for i in idx]
        st, res = sem.solve_batch([meshes[i] for i in idx], [bs[i] for i in idx], xs,
                                  [dict(tol=1e-10, h1=1.0, h2=1.0) for _ in idx])
        assert st == sem.SEM_OK, res
        return xs, res

    alone = [run([i]) for i in range(2)]
    xs, res = run([0, 1])
    for i in range(2):
        assert res[i]["status"] == 0
        assert torch.equal(xs[i], alone[i][0][0])
        assert _residual(probs[i], bs[i].cpu().numpy(), xs[i].cpu().numpy()) <= 1e-10


def test_three_velocity_components_with_per_point_viscosity():
    """One velocity step of Sec. 2, Eq. 4 with a variable viscosity: the three
    components on one mesh in one batch, each equal to its batch of one and
    within the oracle's residual bound for the per-point operator."""
    import torch
    import paper_2109_03592_gb300 as sem
    d = dict(kind="pipe", nc=4, nr=2, nzp=3, N=7, L=2.0)
    m = sem.Mesh(d)
    om = _om(d)
    nu, _ = _fields(om, 91)
    m.set_coefficients(to_gpu(nu), None)
    h1, h2 = 0.05, 30.0  # 1/Re, b0/dt
    P = solver.Problem(om, h1 * nu, h2)
    bs = [to_gpu(P.rhs(forcing.evaluate(om.xyz, forcing.random_modes(410 + c, L=2.0)))) for c in range(3)]
    opts = [dict(tol=1e-10, h1=h1, h2=h2)] * 3
    xs = [torch.zeros_like(b) for b in bs]
    st, res = sem.solve_batch([m, m, m], bs, xs, opts)
    assert st == sem.SEM_OK, res
    for c in range(3):
        x1 = torch.zeros_like(bs[c])
        st1, r1 = sem.solve_batch([m], [bs[c]], [x1], [opts[c]])
        assert st1 == sem.SEM_OK
        assert torch.equal(xs[c], x1) and res[c]["iters"] == r1[0]["iters"]
        assert _residual(P, bs[c].cpu().numpy(), xs[c].cpu().numpy()) <= 1e-10


def test_projection_space_follows_the_coefficients():
    import torch
    import paper_2109_03592_gb300 as sem
    d = CASES["pipe_n5"]
    m = sem.Mesh(d)
    om = _om(d)
    h1, h2 = _fields(om, 71)
    f = [forcing.evaluate(om.xyz, forcing.random_modes(72 + j, L=2.0)) for j in range(3)]
    gp = sem.Projection(m, max_vectors=4, h1=1.0, h2=1.0)
    P0 = solver.Problem(om, 1.0, 1.0)
    for j in range(2):
        x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
        assert gp.solve(to_gpu(P0.rhs(f[j])), x, tol=1e-10)["status"] == 0
    assert gp.size() == 2
    m.set_coefficients(to_gpu(h1), to_gpu(h2))
    P = solver.Problem(om, h1, h2)
    op = projection.Projection(P, 4)
    for j in range(3):
        b = P.rhs(f[j])
        x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
        res = gp.solve(to_gpu(b), x, tol=1e-10)
        ref = op.solve(b, tol=1e-10)
        assert res["status"] == 0
        assert gp.size() == j + 1  # the basis of the old operator was dropped
        assert _residual(P, b, x.cpu().numpy()) <= 1.1e-10
        assert abs(res["iters"] - ref.iters) <= 2, (res, ref.iters)
