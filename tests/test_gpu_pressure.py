"""GPU parity of the staggered P_N - P_{N-2} pressure operators (Sec. 2: GL
pressure points; Sec. 2, Eq. 5: the consistent Poisson operator
E = D B^{-1} D^T) through the C ABI, against the CPU oracle on the same seeded
inputs: small meshes compared in full (several elements, ragged counts,
N = 2 .. 11), the benchmark's E = 262,144 pipe on sampled elements and through
properties that hold at any size."""

import numpy as np
import pytest

from oracle import mesh as omesh, pressure, solver
from sem_inputs import configs

pytestmark = pytest.mark.gpu

TOL = 1e-12  # FP64: relative L2 error bound, as for the FP64 local operator
F_TOL = 1e-13

CASES = {
    "box_n2": dict(kind="box", nx=2, ny=1, nz=3, N=2, lx=1.0, ly=0.5, lz=1.5),     # m = 1: one GL point
    "box_n4": dict(kind="box", nx=2, ny=2, nz=2, N=4),                             # constant null mode
    "box_ragged_n7": dict(kind="box", nx=3, ny=2, nz=1, N=7, lx=1.5, ly=1.0, lz=0.5),
    "pipe_n5": dict(kind="pipe", nc=2, nr=1, nzp=3, N=5, L=3.0),
    "pipe_open_n7": dict(kind="pipe", nc=2, nr=2, nzp=3, N=7, L=2.0, periodic=False),
    "pipe_n11": dict(kind="pipe", nc=1, nr=1, nzp=3, N=11, L=3.0),
}

_cache = {}


def _oracle_mesh(desc):
    if desc["kind"] == "box":
        return omesh.box(desc["nx"], desc["ny"], desc["nz"], desc["N"], desc.get("lx", 1.0), desc.get("ly", 1.0),
                         desc.get("lz", 1.0))
    return omesh.pipe(desc["nc"], desc["nr"], desc["nzp"], desc["N"], L=desc.get("L", 8.0),
                      periodic=desc.get("periodic", True))


def setup(name):
    import paper_2109_03592_gb300 as sem
    if name not in _cache:
        desc = CASES[name]
        _cache[name] = (sem.Mesh(desc), pressure.Pressure(solver.Problem(_oracle_mesh(desc))))
    return _cache[name]


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(CASES))
def test_gl_factors_match_oracle(name):
    m, P = setup(name)
    assert m.pressure_size() == int(np.prod(P.shape))
    F = m.pressure_factors().cpu().numpy()
    Fo = P.F.reshape(F.shape)  # [E, b, a, ...] -> [E, 3 b + a, ...]
    assert np.abs(F - Fo).max() <= F_TOL * np.abs(Fo).max()


@pytest.mark.parametrize("name", list(CASES))
def test_grad_and_div_match_oracle(name):
    import torch
    m, P = setup(name)
    rng = np.random.default_rng(5)
    p = rng.standard_normal(P.shape)
    u = torch.full((3,) + m.shape, float("nan"), dtype=torch.float64, device="cuda")
    m.pressure_grad(to_gpu(p), u)
    assert relerr(u.cpu().numpy(), P.grad(p)) <= TOL
    v = rng.standard_normal((3,) + m.shape)
    q = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
    m.pressure_div(to_gpu(v), q)
    assert relerr(q.cpu().numpy(), P.div(v)) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_consistent_poisson_operator_matches_oracle(name):
    import torch
    m, P = setup(name)
    p = np.random.default_rng(6).standard_normal(P.shape)
    q = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
    work = torch.full((3 * m.n_local,), float("nan"), dtype=torch.float64, device="cuda")
    m.pressure_apply(to_gpu(p), q, work)
    ref = P.E(p)
    assert relerr(q.cpu().numpy(), ref) <= TOL
    # in place (q = p) gives the same bits; a second call reuses the built GL data
    pp = to_gpu(p)
    m.pressure_apply(pp, pp, work)
    assert torch.equal(pp, q)


def test_constant_pressure_is_in_the_null_space_on_the_box():
    import torch
    m, P = setup("box_n4")
    ones = torch.ones(P.shape, dtype=torch.float64, device="cuda")
    q = torch.empty_like(ones)
    m.pressure_apply(ones, q)
    p = torch.from_numpy(np.random.default_rng(8).standard_normal(P.shape)).cuda()
    Ep = torch.empty_like(p)
    m.pressure_apply(p, Ep)
    assert q.abs().max().item() <= 1e-13 * Ep.abs().max().item()


def test_invalid_arguments_rejected():
    import torch
    import paper_2109_03592_gb300 as sem
    m1 = sem.Mesh(dict(kind="box", nx=2, ny=1, nz=1, N=1))
    with pytest.raises(sem.SemError) as ei:
        m1.pressure_size()
    assert ei.value.status == sem.SEM_ERR_INVALID
    m, P = setup("box_n4")
    work = torch.zeros(3 * m.n_local, dtype=torch.float64, device="cuda")
    p = work[: m.pressure_size()]
    q = torch.empty(P.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as ei:
        m.pressure_apply(p, q, work)
    assert ei.value.status == sem.SEM_ERR_INVALID


def test_full_size_pipe_sampled_elements_and_symmetry():
    """E = 262,144, N = 7 (the benchmark's pipe): F, D^T and D on 24 sampled
    elements against the oracle run on those elements alone; E through
    symmetry <q, E p> = <p, E q>, which holds at any size."""
    import torch
    import paper_2109_03592_gb300 as sem
    desc = configs.mesh_desc("pipe262144_n7")
    m = sem.Mesh(desc)
    N, mm = 7, 6
    els = np.sort(np.random.default_rng(9).choice(m.E, 24, replace=False))
    els[0], els[-1] = 0, m.E - 1
    om = omesh.pipe(desc["nc"], desc["nr"], desc["nzp"], N, R=desc["R"], L=desc["L"], a=desc["a"],
                    beta=desc["beta"], periodic=True, elements=els)
    Fo, _ = pressure.div_factors(om)
    F = m.pressure_factors()
    idx = torch.from_numpy(els).cuda()
    Fs = F.index_select(0, idx).cpu().numpy()
    assert np.abs(Fs - Fo.reshape(Fs.shape)).max() <= F_TOL * np.abs(Fo).max()
    del F
    g = torch.Generator(device="cuda").manual_seed(3)
    p = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda", generator=g)
    u = torch.empty((3,) + m.shape, dtype=torch.float64, device="cuda")
    m.pressure_grad(p, u)
    us = u.index_select(1, idx).cpu().numpy()
    ps = p.index_select(0, idx).cpu().numpy()
    assert relerr(us, pressure.grad_local(N, Fo, ps)) <= TOL
    q = torch.empty_like(p)
    m.pressure_div(u, q)
    assert relerr(q.index_select(0, idx).cpu().numpy(), pressure.div_local(N, Fo, us)) <= TOL
    work = u.view(-1)
    r = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda", generator=g)
    Ep = torch.empty_like(p)
    Er = torch.empty_like(p)
    m.pressure_apply(p, Ep, work)
    m.pressure_apply(r, Er, work)
    a, b = torch.dot(r.view(-1), Ep.view(-1)).item(), torch.dot(p.view(-1), Er.view(-1)).item()
    # random fields: the sums cancel to ~1/sqrt(n) of their terms, so the bound
    # is relative to the sum of |terms| (FP64 rounding of E and of the sums)
    scale = torch.dot(r.view(-1).abs(), Ep.view(-1).abs()).item()
    assert abs(a - b) <= 1e-13 * scale
    assert torch.dot(p.view(-1), Ep.view(-1)).item() > 0
    m.close()


SOLVE_CASES = {
    "box_n4": CASES["box_n4"],                                    # exact constant null space
    "pipe_n3": dict(kind="pipe", nc=2, nr=1, nzp=3, N=3, L=1.5),  # curved: near-null constant mode
    "pipe_n4": dict(kind="pipe", nc=1, nr=1, nzp=3, N=4, L=1.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_diagonal_matches_oracle(name):
    """diag(E) (the pressure CG's Jacobi preconditioner) against the oracle's,
    which is itself pinned to the diagonal of the dense E."""
    import torch
    m, P = setup(name)
    d = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
    m.pressure_diag(d)
    assert relerr(d.cpu().numpy(), P.diagonal()) <= TOL


@pytest.mark.parametrize("name", list(SOLVE_CASES))
@pytest.mark.parametrize("precond", ["NONE", "JACOBI"])
def test_pressure_solve_matches_oracle(name, precond):
    """CG on the mean-free space, plain and Jacobi-preconditioned: iteration
    count within 2 of the oracle's, the GPU solution's residual Pm (g - E x)
    recomputed with the oracle's E within the tolerance, mean zero, and close
    to the oracle's solution."""
    import torch
    import paper_2109_03592_gb300 as sem
    desc = SOLVE_CASES[name]
    m = sem.Mesh(desc)
    P = pressure.Pressure(solver.Problem(_oracle_mesh(desc)))
    g = np.random.default_rng(12).standard_normal(P.shape)
    x = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
    r = m.pressure_solve(to_gpu(g), x, tol=1e-10, precond=getattr(sem, "PRECOND_" + precond))
    assert r["status"] == 0, r
    dinv = 1.0 / P.diagonal() if precond == "JACOBI" else None
    xo, it, rel, st = pressure.cg(P, g, tol=1e-10, dinv=dinv)
    assert st == solver.CONVERGED
    assert abs(r["iters"] - it) <= 2, (r["iters"], it)
    assert r["rel_res"] <= 1e-10
    xg = x.cpu().numpy()
    gm = g - g.mean()
    res = g - P.E(xg)
    res = res - res.mean()
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(gm)
    assert abs(xg.sum()) <= 1e-10 * np.abs(xg).sum()
    assert relerr(xg, xo) <= 1e-6
    m.close()


def test_pressure_solve_degenerate_right_hand_sides_and_iteration_cap():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = setup("box_n4")
    for val in (0.0, 3.0):  # zero and constant g: Pm g = 0
        x = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
        r = m.pressure_solve(torch.full(P.shape, val, dtype=torch.float64, device="cuda"), x)
        assert r["status"] == 0 and r["iters"] == 0 and x.abs().max().item() == 0.0
    g = to_gpu(np.random.default_rng(13).standard_normal(P.shape))
    x = torch.empty_like(g)
    r = m.pressure_solve(g, x, maxit=3)
    assert r["status"] == sem.SEM_ERR_NOT_CONVERGED and r["iters"] == 3
    with pytest.raises(sem.SemError) as ei:
        m.pressure_solve(g, g)
    assert ei.value.status == sem.SEM_ERR_INVALID


def test_pressure_solve_on_the_4096_element_pipe():
    """The paper's per-GPU regime (E = 4096, N = 7): the true residual,
    recomputed with the parity-tested operator, meets the tolerance."""
    import torch
    import paper_2109_03592_gb300 as sem
    m = sem.Mesh(configs.mesh_desc("pipe4096_n7"))
    g = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(4))
    x = torch.empty_like(g)
    r = m.pressure_solve(g, x, tol=1e-10)
    assert r["status"] == 0, r
    Ex = torch.empty_like(g)
    m.pressure_apply(x, Ex)
    res = g - Ex
    res -= res.mean()
    gm = g - g.mean()
    assert (res.norm() / gm.norm()).item() <= 2e-10
    assert abs(x.sum().item()) <= 1e-10 * x.abs().sum().item()
    plain = m.pressure_solve(g, torch.empty_like(g), tol=1e-10, precond=sem.PRECOND_NONE)
    assert plain["status"] == 0 and r["iters"] < plain["iters"], (r, plain)
    m.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_operator_matches_oracle(name):
    """The FP32 form of E (factors, basis and fields rounded from FP64) against
    the oracle's FP64 E: the rounding-level bound of FP32 sum factorisation."""
    import torch
    m, P = setup(name)
    p = np.random.default_rng(6).standard_normal(P.shape)
    q = torch.full(P.shape, float("nan"), dtype=torch.float32, device="cuda")
    m.pressure_apply_f32(to_gpu(p).float(), q)
    assert relerr(q.double().cpu().numpy(), P.E(p)) <= 2e-5


@pytest.mark.parametrize("name", list(SOLVE_CASES))
def test_mixed_pressure_solve_meets_the_fp64_tolerance(name):
    """The mixed-precision pressure CG (FP32 E, FP64 reliable updates): the
    GPU solution's residual Pm (g - E x) recomputed with the oracle's FP64 E
    meets 1e-10, the solution is mean-free and matches the FP64 solve."""
    import torch
    import paper_2109_03592_gb300 as sem
    desc = SOLVE_CASES[name]
    m = sem.Mesh(desc)
    P = pressure.Pressure(solver.Problem(_oracle_mesh(desc)))
    g = np.random.default_rng(12).standard_normal(P.shape)
    x = torch.full(P.shape, float("nan"), dtype=torch.float64, device="cuda")
    r = m.pressure_solve(to_gpu(g), x, tol=1e-10, prec=sem.MIXED)
    assert r["status"] == 0, r
    assert r["rel_res"] <= 1e-10 and r["outer_iters"] >= 1
    xg = x.cpu().numpy()
    gm = g - g.mean()
    res = g - P.E(xg)
    res = res - res.mean()
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(gm)
    assert abs(xg.sum()) <= 1e-10 * np.abs(xg).sum()
    x64 = torch.empty_like(x)
    r64 = m.pressure_solve(to_gpu(g), x64, tol=1e-10)
    assert relerr(xg, x64.cpu().numpy()) <= 1e-6
    assert r["iters"] <= 2 * r64["iters"] + 20, (r, r64)
    m.close()


def test_mixed_pressure_solve_on_the_4096_element_pipe():
    import torch
    import paper_2109_03592_gb300 as sem
    m = sem.Mesh(configs.mesh_desc("pipe4096_n7"))
    g = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(4))
    x = torch.empty_like(g)
    r = m.pressure_solve(g, x, tol=1e-10, prec=sem.MIXED)
    assert r["status"] == 0, r
    Ex = torch.empty_like(g)
    m.pressure_apply(x, Ex)
    res = g - Ex
    res -= res.mean()
    gm = g - g.mean()
    assert (res.norm() / gm.norm()).item() <= 2e-10
    m.close()
