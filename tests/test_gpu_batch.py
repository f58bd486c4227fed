"""Batched mixed-precision solves (sem_pcg_solve_batch): one CUDA graph of
batched kernels advances all requests of one order; each result equals the
result of a batch of one, and meets the FP64 residual bound of the oracle."""

import numpy as np
import pytest

from oracle import mesh as omesh, solver
from sem_inputs import forcing

pytestmark = pytest.mark.gpu

REQS = [
    (dict(kind="box", nx=3, ny=3, nz=3, N=5), 0.0),
    (dict(kind="pipe", nc=2, nr=1, nzp=3, N=5, L=3.0), 2.0),
    (dict(kind="box", nx=2, ny=3, nz=5, N=5), 0.5),
    (dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0), 0.0),
    (dict(kind="box", nx=1, ny=1, nz=1, N=5), 0.0),          # single element
    (dict(kind="pipe", nc=2, nr=2, nzp=5, N=5, L=4.0), 10.0),
]


def _om(d):
    if d["kind"] == "box":
        return omesh.box(d["nx"], d["ny"], d["nz"], d["N"])
    return omesh.pipe(d["nc"], d["nr"], d["nzp"], d["N"], L=d["L"])


@pytest.fixture(scope="module")
def problems():
    import torch
    import paper_2109_03592_gb300 as sem
    out = []
    for i, (d, h2) in enumerate(REQS):
        om = _om(d)
        P = solver.Problem(om, 1.0, h2)
        b = P.rhs(forcing.evaluate(om.xyz, forcing.random_modes(200 + i, L=d.get("L", 1.0))))
        out.append((sem.Mesh(d), P, torch.from_numpy(b).cuda(), h2))
    return out


def _run(problems, idx):
    import torch
    import paper_2109_03592_gb300 as sem
    meshes = [problems[i][0] for i in idx]
    bs = [problems[i][2] for i in idx]
    xs = [torch.zeros_like(b) for b in bs]
    opts = [dict(tol=1e-10, h1=1.0, h2=problems[i][3]) for i in idx]
    st, res = sem.solve_batch(meshes, bs, xs, opts)
    assert st == sem.SEM_OK, res
    return xs, res


def test_batch_equals_batch_of_one_and_meets_residual(problems):
    alone = [_run(problems, [i]) for i in range(len(problems))]
    xs, res = _run(problems, list(range(len(problems))))
    for i, (m, P, b, h2) in enumerate(problems):
        assert res[i]["status"] == 0
        assert np.array_equal(xs[i].cpu().numpy(), alone[i][0][0].cpu().numpy()), i
        assert res[i]["iters"] == alone[i][1][0]["iters"]
        bn = b.cpu().numpy()
        r = bn - P.A(xs[i].cpu().numpy())
        assert np.sqrt(P.dot(r, r) / P.dot(bn, bn)) <= 1e-10
        ref = solver.pcg_mixed_reliable(P, bn, tol=1e-10, delta=0.1)  # the batched solves' default
        assert abs(res[i]["iters"] - ref.iters) <= 0.1 * ref.iters + 3, (i, res[i], ref.iters)


def test_batch_more_requests_than_slots(problems):
    """40 requests through 32 slots: later ones join as earlier ones finish."""
    import torch
    import paper_2109_03592_gb300 as sem
    meshes, bs, xs, opts = [], [], [], []
    base = dict(kind="box", nx=2, ny=2, nz=2, N=3)
    P = solver.Problem(omesh.box(2, 2, 2, 3))
    for k in range(40):
        meshes.append(sem.Mesh(base))
        b = P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(300 + k)))
        bs.append(torch.from_numpy(b).cuda())
        xs.append(torch.zeros_like(bs[-1]))
        opts.append(dict(tol=1e-10))
    st, res = sem.solve_batch(meshes, bs, xs, opts)
    assert st == sem.SEM_OK
    for k in range(40):
        bn = bs[k].cpu().numpy()
        r = bn - P.A(xs[k].cpu().numpy())
        assert res[k]["status"] == 0 and np.sqrt(P.dot(r, r) / P.dot(bn, bn)) <= 1e-10


def test_three_right_hand_sides_on_one_mesh():
    """The three velocity components of a Helmholtz step (h2 = b0/dt) on one
    mesh in one batch: each equals its batch of one and meets the residual."""
    import torch
    import paper_2109_03592_gb300 as sem
    d = dict(kind="pipe", nc=4, nr=2, nzp=3, N=7, L=2.0)
    m = sem.Mesh(d)
    P = solver.Problem(_om(d), 0.05, 30.0)  # h1 = 1/Re, h2 = b0/dt
    bs = [torch.from_numpy(P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(400 + c, L=2.0)))).cuda()
          for c in range(3)]
    opts = [dict(tol=1e-10, h1=0.05, h2=30.0)] * 3
    xs = [torch.zeros_like(b) for b in bs]
    st, res = sem.solve_batch([m, m, m], bs, xs, opts)
    assert st == sem.SEM_OK, res
    for c in range(3):
        x1 = torch.zeros_like(bs[c])
        st1, r1 = sem.solve_batch([m], [bs[c]], [x1], [opts[c]])
        assert st1 == sem.SEM_OK
        assert torch.equal(xs[c], x1) and res[c]["iters"] == r1[0]["iters"]
        bn = bs[c].cpu().numpy()
        r = bn - P.A(xs[c].cpu().numpy())
        assert np.sqrt(P.dot(r, r) / P.dot(bn, bn)) <= 1e-10
    m.close()


def test_batch_rejects_mixed_orders_and_even_N(problems):
    import torch
    import paper_2109_03592_gb300 as sem
    m5 = problems[0][0]
    m7 = sem.Mesh(dict(kind="box", nx=2, ny=2, nz=2, N=7))
    b5 = problems[0][2]
    b7 = torch.zeros(m7.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.solve_batch([m5, m7], [b5, b7], [torch.zeros_like(b5), torch.zeros_like(b7)], tol=1e-10)
    m4 = sem.Mesh(dict(kind="box", nx=2, ny=2, nz=2, N=4))
    b4 = torch.zeros(m4.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        sem.solve_batch([m4], [b4], [torch.zeros_like(b4)], tol=1e-10)
