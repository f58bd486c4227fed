"""GPU tests of the request server (sem_server_*): continuous admission of
Poisson/Helmholtz solves of different sizes and orders, overlapping on one
GPU, with each result identical alone and in the mix."""

import time

import numpy as np
import pytest

from oracle import mesh as omesh, solver
from sem_inputs import forcing

pytestmark = pytest.mark.gpu

REQS = [
    (dict(kind="box", nx=3, ny=3, nz=3, N=5), 0.0),
    (dict(kind="pipe", nc=2, nr=1, nzp=3, N=5, L=3.0), 2.0),
    (dict(kind="box", nx=2, ny=3, nz=4, N=7), 0.5),
    (dict(kind="pipe", nc=4, nr=1, nzp=3, N=3, L=2.0), 0.0),
    (dict(kind="box", nx=4, ny=4, nz=2, N=3), 10.0),
    (dict(kind="pipe", nc=2, nr=2, nzp=4, N=7, L=4.0), 0.0),
]


def _oracle_mesh(d):
    if d["kind"] == "box":
        return omesh.box(d["nx"], d["ny"], d["nz"], d["N"])
    return omesh.pipe(d["nc"], d["nr"], d["nzp"], d["N"], L=d["L"])


def _forcing(d, seed):
    m = _oracle_mesh(d)
    return m, forcing.evaluate(m.xyz, forcing.random_modes(seed, L=d.get("L", 1.0)))


@pytest.fixture(scope="module")
def inputs():
    return [(d, h2, *_forcing(d, 100 + i)) for i, (d, h2) in enumerate(REQS)]


def _solve_all(srv, inputs, prec):
    import paper_2109_03592_gb300 as sem
    ids = [srv.submit(d, f, tol=1e-10, h1=1.0, h2=h2, prec=prec) for d, h2, m, f in inputs]
    out = []
    for rid, (d, h2, m, f) in zip(ids, inputs):
        st, x, res = srv.poll(rid, timeout_ms=-1, n_local=f.size)
        assert st == sem.SEM_OK, (st, res)
        out.append((x, res))
    return out


@pytest.mark.parametrize("prec,batch", [("mixed", True), ("mixed", False), ("fp64", True)])
def test_results_same_alone_and_in_the_mix(inputs, prec, batch):
    """Mixed precision with batching: odd-order requests share per-order
    batches (one graph of batched kernels); without batching, and for FP64,
    each request runs on its slot's stream.  Either way a request's result is
    bitwise the same alone and among 11 others."""
    import paper_2109_03592_gb300 as sem
    pr = sem.MIXED if prec == "mixed" else sem.FP64
    alone = []
    srv1 = sem.Server(max_slots=1, batch=batch)
    for item in inputs:  # one request at a time on an idle server
        alone += _solve_all(srv1, [item], pr)
    srv1.close()
    srv = sem.Server(max_slots=4, batch=batch)
    mixed = _solve_all(srv, inputs + inputs, pr)  # 12 requests, 4 in flight
    st = srv.stats()
    srv.close()
    assert st["completed"] == 12 and st["rejected"] == 0
    for k, (d, h2, m, f) in enumerate(inputs):
        for x, res in (mixed[k], mixed[k + len(inputs)]):
            assert np.array_equal(x, alone[k][0]), (k, d)
            assert res["iters"] == alone[k][1]["iters"]
        P = solver.Problem(m, 1.0, h2)
        b = P.rhs(f)
        r = b - P.A(alone[k][0].reshape(P.shape))
        assert np.sqrt(P.dot(r, r) / P.dot(b, b)) <= 1.1e-10


def test_admission_queue_cancel_and_timeout(inputs):
    import paper_2109_03592_gb300 as sem
    d, h2, m, f = inputs[0]
    # a budget smaller than one request's footprint: rejected at submit
    srv = sem.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    with pytest.raises(sem.SemError) as ei:
        srv.submit(d, f)
    assert ei.value.status == sem.SEM_ERR_OOM
    assert srv.stats()["rejected"] == 1
    srv.close()
    # one slot solving every request itself (no batching), a short queue:
    # later submissions wait, the queue bounds them
    srv = sem.Server(max_slots=1, max_queue=3, batch=False)
    big = dict(kind="pipe", nc=4, nr=2, nzp=24, N=7, L=8.0)
    fbig = np.zeros(4 * 12 * 24 * 512)
    fbig[:] = 1.0
    first = srv.submit(big, fbig, prec=sem.MIXED)
    t0 = time.perf_counter()
    while srv.stats()["running"] == 0 and time.perf_counter() - t0 < 10:
        time.sleep(0.001)
    queued = [srv.submit(d, f) for _ in range(3)]
    with pytest.raises(sem.SemError) as ei:
        srv.submit(d, f)
    assert ei.value.status in (sem.SEM_ERR_BUSY,)
    st, x, res = srv.poll(queued[-1], timeout_ms=0)
    assert st == sem.SEM_ERR_TIMEOUT and x is None
    assert srv.cancel(queued[-1]) == sem.SEM_OK
    st, x, res = srv.poll(queued[-1], timeout_ms=1000)
    assert st == sem.SEM_ERR_CANCELLED
    for rid in [first] + queued[:-1]:
        st, x, res = srv.poll(rid, timeout_ms=-1)
        assert st == sem.SEM_OK
    with pytest.raises(sem.SemError) as ei:
        srv.poll(first, timeout_ms=0)
    assert ei.value.status == sem.SEM_ERR_NOT_FOUND
    s = srv.stats()
    assert s["cancelled"] == 1 and s["completed"] == 3 and s["running"] == 0 and s["hbm_in_use"] == 0
    srv.close()


def test_request_stream_latency(inputs):
    """A short Poisson-arrival stream: requests are admitted while others run
    (continuous batching), all finish, and p50/p99 latencies are finite."""
    import paper_2109_03592_gb300 as sem
    from sem_inputs import serving
    stream = serving.request_stream(seed=4, count=16, rate=40.0, log2_e=(6.0, 9.0), orders=(3, 5))
    srv = sem.Server(max_slots=4)
    t0 = time.perf_counter()
    pending = {}
    for req in stream:
        now = time.perf_counter() - t0
        if req["arrival"] > now:
            time.sleep(req["arrival"] - now)
        d = req["desc"]
        n = d["N"] + 1
        E = d["nx"] * d["ny"] * d["nz"] if d["kind"] == "box" else d["nc"] * (d["nc"] + 4 * d["nr"]) * d["nzp"]
        f = np.random.default_rng(req["seed"]).standard_normal(E * n ** 3)
        rid = srv.submit(d, f, tol=1e-10, h1=1.0, h2=req["h2"], prec=sem.MIXED)
        pending[rid] = (time.perf_counter(), E * n ** 3)
    lat = []
    for rid, (ts, nl) in pending.items():
        st, x, res = srv.poll(rid, timeout_ms=-1, n_local=nl)
        assert st == sem.SEM_OK, res
        lat.append(time.perf_counter() - ts)
        assert res["rel_res"] <= 1e-10
    srv.close()
    assert len(lat) == 16 and np.percentile(lat, 99) < 60.0
