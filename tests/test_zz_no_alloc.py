"""sem_pcg_solve_noalloc: the FP64 solve for callers that cannot allocate
device memory (their memory belongs to a fixed pool or another allocator, or
an allocation's latency and implicit synchronisation are not acceptable).

Its scratch lives in the library's fixed device array.  These tests compare
it, through the C ABI, with sem_pcg_solve on the same inputs, for two calls
in a row (the array keeps the previous call's contents), and check that a
mesh above the size limit is rejected.  The file is collected last on
purpose: the first test must also work when it is the first call of a fresh
process, and after every other test has run."""

import numpy as np
import pytest

from oracle import mesh as omesh, solver
from sem_inputs import forcing

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-10


def _case():
    import torch
    import paper_2109_03592_gb300 as sem
    desc = dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0)
    m = sem.Mesh(desc)
    P = solver.Problem(omesh.pipe(4, 2, 3, 5, L=2.0), 1.0, 0.5)
    b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(9, L=2.0)))
    return m, P, torch.from_numpy(b).cuda()


def test_noalloc_solve_matches_pcg_solve_twice():
    import torch
    m, P, b = _case()
    assert m.n_local <= 1 << 18
    x_ref = torch.zeros_like(b)
    ref = m.solve(b, x_ref, tol=SOLVE_TOL, h1=1.0, h2=0.5)
    assert ref["status"] == 0
    for call in range(2):
        x = torch.zeros_like(b)
        res = m.solve_noalloc(b, x, tol=SOLVE_TOL, h1=1.0, h2=0.5)
        assert res["status"] == 0, (call, res)
        assert abs(res["iters"] - ref["iters"]) <= 2, (call, res, ref)
        xs, xr = x.cpu().numpy(), x_ref.cpu().numpy()
        err = np.sqrt(P.dot(xs - xr, xs - xr) / P.dot(xr, xr))
        assert err < 1e-8, (call, err)
        r = b.cpu().numpy() - P.A(xs)
        bn = b.cpu().numpy()
        assert np.sqrt(P.dot(r, r) / P.dot(bn, bn)) <= 1.1e-10


@pytest.mark.parametrize("kernel", ["df", "native"])
def test_noalloc_reports_the_true_residual(monkeypatch, kernel):
    """The reported rel_res is the true residual ||b - A x|| / ||b||, formed
    after the CG recurrences stop; the oracle's FP64 operator recomputes it.
    With the double-float CG operator forced, the recurrence alone would not
    show whether the true residual meets the tolerance."""
    import paper_2109_03592_gb300 as sem
    monkeypatch.setenv("SEM_FP64_KERNEL", kernel)
    m, P, b = _case()
    assert m.fp64_double_float() == (kernel == "df")
    import torch
    bn = b.cpu().numpy()
    for call in range(2):
        x = torch.zeros_like(b)
        res = m.solve_noalloc(b, x, tol=SOLVE_TOL, h1=1.0, h2=0.5)
        assert res["status"] == 0, (call, res)
        r = bn - P.A(x.cpu().numpy())
        true_rel = np.sqrt(P.dot(r, r) / P.dot(bn, bn))
        assert true_rel <= 1.05e-10, (call, true_rel)
        assert abs(res["rel_res"] - true_rel) <= 1e-3 * true_rel + 1e-15, (call, res, true_rel)
    # a starting guess that already meets the tolerance: no iteration, the same residual
    res2 = m.solve_noalloc(b, x, tol=SOLVE_TOL, h1=1.0, h2=0.5)
    assert res2["status"] == 0 and res2["iters"] == 0, res2
    assert abs(res2["rel_res"] - res["rel_res"]) <= 1e-3 * res["rel_res"], (res2, res)


def test_noalloc_rejects_large_mesh_and_other_precisions():
    import torch
    import paper_2109_03592_gb300 as sem
    big = sem.Mesh(dict(kind="box", nx=9, ny=8, nz=8, N=7))  # 589,824 local points
    assert big.n_local > sem.sem.NOALLOC_MAX_POINTS
    b = torch.zeros(big.shape, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(sem.SemError) as ei:
        big.solve_noalloc(b, x)
    assert ei.value.status == sem.SEM_ERR_INVALID
    m, P, b = _case()
    x = torch.zeros_like(b)
    with pytest.raises(sem.SemError) as ei:
        m.solve_noalloc(b, x, prec=sem.MIXED)
    assert ei.value.status == sem.SEM_ERR_INVALID
