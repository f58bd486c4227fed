"""The overlapping Schwarz preconditioner on the GPU (sem_schwarz_*, Sec. 2,
Eq. 6) against the oracle's (oracle/schwarz.py): M^{-1} r element by element
in FP64 (1e-12) and FP32, and Schwarz-PCG iteration counts and residuals."""

import numpy as np
import pytest

from oracle import mesh as omesh, schwarz, solver
from sem_inputs import forcing

pytestmark = pytest.mark.gpu

CASES = {
    "box222_n3": (dict(kind="box", nx=2, ny=2, nz=2, N=3), lambda: omesh.box(2, 2, 2, 3)),
    "box322_n7": (dict(kind="box", nx=3, ny=2, nz=2, N=7, lx=1.5, ly=1.0, lz=0.8),
                  lambda: omesh.box(3, 2, 2, 7, lx=1.5, ly=1.0, lz=0.8)),
    "pipe213_n3": (dict(kind="pipe", nc=2, nr=1, nzp=3, N=3, L=1.5), lambda: omesh.pipe(2, 1, 3, 3, L=1.5)),
    "pipe423_n5": (dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0), lambda: omesh.pipe(4, 2, 3, 5, L=2.0)),
    "pipe213_n8_open": (dict(kind="pipe", nc=2, nr=1, nzp=3, N=8, L=1.5, periodic=False),
                        lambda: omesh.pipe(2, 1, 3, 8, L=1.5, periodic=False)),
}


def _make(name, h2=0.0):
    import paper_2109_03592_gb300 as sem
    desc, om = CASES[name]
    return sem.Mesh(desc), solver.Problem(om(), 1.0, h2)


def _residual_field(P, seed):
    """A continuous, masked field like a CG residual."""
    v = np.random.default_rng(seed).standard_normal(P.shape)
    return P.mask * P.gs(v)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("coarse", [True, False])
@pytest.mark.parametrize("h2", [0.0, 2.5])
def test_apply_fp64_matches_oracle(name, coarse, h2):
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make(name, h2)
    sw = sem.Schwarz(m, 1.0, h2, coarse=coarse)
    info = sw.info()
    assert info["coarse"] == coarse
    ref_sw = schwarz.Schwarz(P, coarse=coarse)
    for seed in (1, 2):
        r = _residual_field(P, seed)
        z = torch.empty(m.shape, dtype=torch.float64, device="cuda")
        sw.apply(torch.from_numpy(r).cuda(), z)
        ref = ref_sw.apply(r)
        got = z.cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-12, (name, coarse, h2, rel)
    sw.close()
    m.close()


@pytest.mark.parametrize("name", ["box322_n7", "pipe423_n5"])
def test_apply_fp32_matches_oracle(name):
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make(name)
    sw = sem.Schwarz(m)
    ref_sw = schwarz.Schwarz(P)
    r = _residual_field(P, 3)
    z = torch.empty(m.shape, dtype=torch.float32, device="cuda")
    sw.apply(torch.from_numpy(r).float().cuda(), z, prec=sem.FP32)
    ref = ref_sw.apply(r)
    rel = np.linalg.norm(z.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel <= 2e-5, rel
    sw.close()
    m.close()


def _rhs(P, seed, L):
    return P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(seed, L=L)))


def _rel_residual(P, b, x):
    r = b - P.A(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


@pytest.mark.parametrize("name", ["box322_n7", "pipe423_n5", "pipe213_n8_open"])
@pytest.mark.parametrize("coarse", [True, False])
def test_fp64_solve_matches_oracle(name, coarse):
    """FP64 Schwarz-PCG: iterations within 2 of the oracle's PCG with its own
    preconditioner, and the GPU solution's residual recomputed by the oracle."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make(name)
    b = _rhs(P, 11, CASES[name][0].get("L", 1.0))
    ref = schwarz.pcg(P, b, schwarz.Schwarz(P, coarse=coarse).apply, tol=1e-10)
    sw = sem.Schwarz(m, coarse=coarse)
    x = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    res = sw.solve(torch.from_numpy(b).cuda(), x, tol=1e-10)
    assert res["status"] == 0, res
    assert abs(res["iters"] - ref.iters) <= 2, (res, ref.iters)
    assert _rel_residual(P, b, x.cpu().numpy()) <= 1.1e-10
    sw.close()
    m.close()


@pytest.mark.parametrize("name", ["box322_n7", "pipe423_n5"])
@pytest.mark.parametrize("h2", [0.0, 2.5])
def test_mixed_solve_residual(name, h2):
    """FP32 Schwarz-PCG with FP64 reliable updates: the residual recomputed by
    the oracle meets 1e-10, in about as many iterations as the FP64 solve."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make(name, h2)
    b = _rhs(P, 12, CASES[name][0].get("L", 1.0))
    sw = sem.Schwarz(m, 1.0, h2)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    r64 = sw.solve(bt, x, tol=1e-10, h2=h2)
    x.zero_()
    res = sw.solve(bt, x, tol=1e-10, h2=h2, prec=sem.MIXED)
    assert res["status"] == 0, res
    assert _rel_residual(P, b, x.cpu().numpy()) <= 1e-10
    assert res["iters"] <= 1.5 * r64["iters"] + 10, (res, r64)
    # the same solve again: bitwise the same iterate (deterministic reductions, captured graphs)
    x2 = torch.zeros_like(bt)
    res2 = sw.solve(bt, x2, tol=1e-10, h2=h2, prec=sem.MIXED)
    assert res2["iters"] == res["iters"] and torch.equal(x, x2)
    sw.close()
    m.close()


def test_fewer_iterations_than_jacobi():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make("pipe423_n5")
    b = torch.from_numpy(_rhs(P, 13, 2.0)).cuda()
    x = torch.zeros_like(b)
    jac = m.solve(b, x, tol=1e-10)
    sw = sem.Schwarz(m)
    x.zero_()
    res = sw.solve(b, x, tol=1e-10)
    assert res["status"] == 0 and jac["status"] == 0
    assert res["iters"] < 0.5 * jac["iters"], (res, jac)
    sw.close()
    m.close()


def test_invalid_arguments():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make("box222_n3")
    with pytest.raises(sem.SemError) as ei:
        sem.Schwarz(m, 0.0, 0.0)
    assert ei.value.status == sem.SEM_ERR_INVALID
    sw = sem.Schwarz(m, 1.0, 0.0)
    b = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(sem.SemError) as ei:  # another operator than the preconditioner's
        sw.solve(b, x, h2=1.0, check=True)
    assert ei.value.status == sem.SEM_ERR_INVALID
    res = sw.solve(b, x, check=True)  # b = 0: x = 0 at once
    assert res["iters"] == 0 and float(x.abs().max()) == 0.0
    # per-point coefficients: the separable local solves take scalars
    h1 = torch.ones(m.shape, dtype=torch.float64, device="cuda")
    m.set_coefficients(h1, None)
    with pytest.raises(sem.SemError) as ei:
        sem.Schwarz(m)
    assert ei.value.status == sem.SEM_ERR_INVALID
    with pytest.raises(sem.SemError) as ei:  # built before the change: stale
        sw.apply(b, x)
    assert ei.value.status == sem.SEM_ERR_INVALID
    sw.close()
    m.close()


@pytest.mark.parametrize("name", ["box322_n7", "pipe423_n5"])
def test_fp64_solve_with_the_fp32_preconditioner(name):
    """FP64 CG with z = M32 float(r): the oracle's residual meets 1e-10, in
    about as many iterations as with the FP64 preconditioner."""
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _make(name)
    b = _rhs(P, 14, CASES[name][0].get("L", 1.0))
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    ref = sem.Schwarz(m).solve(bt, x, tol=1e-10)
    sw = sem.Schwarz(m, fp32_precond=True)
    x.zero_()
    res = sw.solve(bt, x, tol=1e-10)
    assert res["status"] == 0, res
    assert _rel_residual(P, b, x.cpu().numpy()) <= 1.1e-10
    assert abs(res["iters"] - ref["iters"]) <= max(3, ref["iters"] // 10), (res, ref)
    sw.close()
    m.close()
