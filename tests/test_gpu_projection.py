"""GPU projection onto previous solutions (sem_proj_*) against the oracle's
projection (oracle/projection.py) on the same sequence of right-hand sides."""

import numpy as np
import pytest

from oracle import mesh as omesh, projection, solver
from sem_inputs import forcing

pytestmark = pytest.mark.gpu

DESC = dict(kind="pipe", nc=4, nr=2, nzp=3, N=5, L=2.0)


def _setup(h2=0.0):
    import paper_2109_03592_gb300 as sem
    m = sem.Mesh(DESC)
    P = solver.Problem(omesh.pipe(DESC["nc"], DESC["nr"], DESC["nzp"], DESC["N"], L=DESC["L"]), 1.0, h2)
    return m, P


def _rhs(P, seed):
    return P.rhs(forcing.evaluate(P.mesh.xyz, forcing.random_modes(seed, L=2.0)))


def _sequence(P, k):
    """Slowly varying right-hand sides (as over time steps)."""
    f0 = forcing.evaluate(P.mesh.xyz, forcing.random_modes(5, L=2.0))
    f1 = forcing.evaluate(P.mesh.xyz, forcing.random_modes(6, L=2.0))
    return [P.rhs(f0 * (1.0 + 0.05 * j) + 0.1 * np.sin(0.4 * j) * f1) for j in range(k)]


def _residual(P, b, x):
    r = b - P.A(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


@pytest.mark.parametrize("h2", [0.0, 3.0])
def test_sequence_matches_oracle(h2):
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _setup(h2)
    gp = sem.Projection(m, max_vectors=4, h1=1.0, h2=h2)
    op = projection.Projection(P, 4)
    for j, b in enumerate(_sequence(P, 7)):
        x = torch.full(m.shape, float("nan"), dtype=torch.float64, device="cuda")  # output only
        res = gp.solve(torch.from_numpy(b).cuda(), x, tol=1e-10)
        ref = op.solve(b, tol=1e-10)
        assert res["status"] == 0
        assert _residual(P, b, x.cpu().numpy()) <= 1.1e-10
        assert abs(res["iters"] - ref.iters) <= 2, (j, res["iters"], ref.iters)
        assert gp.size() == len(op.X)  # restarts at the same step (max_vectors = 4)
    gp.close()
    m.close()


def test_right_hand_sides_in_the_span():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _setup()
    gp = sem.Projection(m, max_vectors=8)
    bs = [torch.from_numpy(_rhs(P, 60 + s)).cuda() for s in range(3)]
    xs = []
    for b in bs:
        x = torch.empty(m.shape, dtype=torch.float64, device="cuda")
        assert gp.solve(b, x, tol=1e-11)["status"] == 0
        xs.append(x)
    assert gp.size() == 3
    x = torch.empty_like(xs[0])
    res = gp.solve(bs[1], x, tol=1e-9)
    assert res["iters"] == 0 and res["status"] == 0
    assert float((x - xs[1]).norm() / xs[1].norm()) <= 1e-9
    res = gp.solve(2.0 * bs[0] - 0.5 * bs[2], x, tol=1e-9)
    assert res["iters"] == 0
    assert gp.size() == 3  # nothing new to add
    gp.reset()
    assert gp.size() == 0
    res = gp.solve(bs[1], x, tol=1e-9)
    assert res["iters"] > 10  # no basis: a full solve again
    gp.close()
    m.close()


def test_mixed_precision_and_fewer_iterations():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _setup()
    gp = sem.Projection(m, max_vectors=8)
    with_p = without = 0
    for b in _sequence(P, 6):
        bt = torch.from_numpy(b).cuda()
        x = torch.empty(m.shape, dtype=torch.float64, device="cuda")
        r = gp.solve(bt, x, tol=1e-10, prec=sem.MIXED)
        assert r["status"] == 0 and _residual(P, b, x.cpu().numpy()) <= 1e-10
        with_p += r["iters"]
        x.zero_()
        without += m.solve(bt, x, tol=1e-10, prec=sem.MIXED)["iters"]
    assert with_p < 0.5 * without
    gp.close()
    m.close()


def test_bad_arguments():
    import torch
    import paper_2109_03592_gb300 as sem
    m, P = _setup()
    with pytest.raises(sem.SemError):
        sem.Projection(m, max_vectors=0)
    with pytest.raises(sem.SemError):
        sem.Projection(m, max_vectors=17)
    gp = sem.Projection(m, max_vectors=2, h1=1.0, h2=0.0)
    b = torch.from_numpy(_rhs(P, 3)).cuda()
    x = torch.empty_like(b)
    with pytest.raises(sem.SemError):
        gp.solve(b, x, h2=1.0)  # not the space's operator
    gp.close()
    m.close()
