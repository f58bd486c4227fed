"""The multi-rank split of QQ^T (sem_gs_halo), emulated with two gloo ranks on
the CPU: each rank sums the nodes whose copies are all its own, exchanges its
copy values of the halo nodes, sums every halo node's copies in the listed
order, and the ranks' vectors together equal the oracle's single-rank QQ^T
bit for bit."""

import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DESC = dict(kind="pipe", nc=2, nr=1, nzp=4, N=3, L=2.0)  # periodic in z: both slab faces are shared


def _setup():
    sys.path.insert(0, ROOT)
    import paper_2109_03592_gb300 as sem
    vert = sem.mesh_vertices(DESC)
    E, N = vert.shape[0], DESC["N"]
    glo, n_global = sem.topology_numbering(E, N, vert)
    return sem, vert, E, N, np.asarray(glo), int(n_global)


def _field(E, n3):
    return np.random.default_rng(11).standard_normal(E * n3).astype(np.float64)


def _reference(v, glo, n_global):
    from oracle import numbering
    return numbering.gs(v.copy(), glo, n_global)


def _rank_qqt(sem, vert, E, N, glo, elem_rank, rank, v_all, exchange):
    """QQ^T on one rank's local vector with the halo exchange done by `exchange`
    (list of this rank's halo copy values -> list of every rank's)."""
    n3 = (N + 1) ** 3
    mine = np.nonzero(elem_rank == rank)[0]
    local = np.concatenate([v_all[e * n3:(e + 1) * n3] for e in mine])
    gloc = np.concatenate([glo[e * n3:(e + 1) * n3] for e in mine])
    gid, ptr, crank, cloc = sem.gs_halo(E, N, vert, elem_rank, rank)
    halo = set(gid.tolist())
    out = local.copy()
    # interior nodes: every copy is on this rank; sum in ascending local index
    order = np.argsort(gloc, kind="stable")
    g_sorted = gloc[order]
    starts = np.r_[0, np.nonzero(np.diff(g_sorted))[0] + 1]
    ends = np.r_[starts[1:], g_sorted.size]
    for s0, s1 in zip(starts, ends):
        if int(g_sorted[s0]) in halo:
            continue
        acc = local[order[s0]]
        for q in range(s0 + 1, s1):
            acc = acc + local[order[q]]
        out[order[s0:s1]] = acc
    # halo nodes: send my copy values, receive everyone's, sum in the listed order
    send = [float(local[cloc[c]]) for c in range(crank.size) if crank[c] == rank]
    received = exchange(send)  # received[r] = rank r's values, in the same list order restricted to r
    cursor = {r: 0 for r in range(len(received))}
    vals = np.empty(crank.size)
    for c in range(crank.size):
        r = int(crank[c])
        vals[c] = received[r][cursor[r]]
        cursor[r] += 1
    for k in range(gid.size):
        acc = vals[ptr[k]]
        for c in range(ptr[k] + 1, ptr[k + 1]):
            acc = acc + vals[c]
        for c in range(ptr[k], ptr[k + 1]):
            if crank[c] == rank:
                out[cloc[c]] = acc
    return mine, out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sem, vert, E, N, glo, n_global = _setup()
    n3 = (N + 1) ** 3
    elem_rank = (np.arange(E) * world // E).astype(np.int32)  # contiguous slabs of elements
    v = _field(E, n3)

    def exchange(send):
        got = [None] * world
        dist.all_gather_object(got, send)
        return got

    mine, out = _rank_qqt(sem, vert, E, N, glo, elem_rank, rank, v, exchange)
    parts = [None] * world
    dist.all_gather_object(parts, (mine.tolist(), out.tolist()))
    if rank == 0:
        full = np.empty(E * n3)
        for els, vals in parts:
            vals = np.asarray(vals)
            for i, e in enumerate(els):
                full[e * n3:(e + 1) * n3] = vals[i * n3:(i + 1) * n3]
        ref = _reference(v, glo, n_global)
        q.put(bool(np.array_equal(full, ref)))
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_rank_gs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 500
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    assert q.get(timeout=10) is True


def test_halo_structure():
    sem, vert, E, N, glo, n_global = _setup()
    n3 = (N + 1) ** 3
    elem_rank = (np.arange(E) * 2 // E).astype(np.int32)
    for rank in (0, 1):
        gid, ptr, crank, cloc = sem.gs_halo(E, N, vert, elem_rank, rank)
        assert gid.size > 0 and np.all(np.diff(gid) > 0)
        mine = np.nonzero(elem_rank == rank)[0]
        for k in range(gid.size):
            ranks = crank[ptr[k]:ptr[k + 1]]
            assert rank in ranks and np.any(ranks != rank)
            # the copies are exactly the global node's local points, in ascending order
            pts = np.nonzero(glo == gid[k])[0]
            assert ptr[k + 1] - ptr[k] == pts.size
            for c, l in zip(range(ptr[k], ptr[k + 1]), pts):
                e = l // n3
                assert crank[c] == elem_rank[e]
                pos = np.searchsorted(np.nonzero(elem_rank == elem_rank[e])[0], e)
                assert cloc[c] == pos * n3 + l % n3
        # the halo is every node this rank shares: its other nodes lie on it alone
        own = set(np.concatenate([glo[e * n3:(e + 1) * n3] for e in mine]).tolist())
        others = set(np.concatenate([glo[e * n3:(e + 1) * n3] for e in np.nonzero(elem_rank != rank)[0]]).tolist())
        assert set(gid.tolist()) == own & others


def test_one_rank_has_no_halo():
    sem, vert, E, N, glo, n_global = _setup()
    gid, ptr, crank, cloc = sem.gs_halo(E, N, vert, np.zeros(E, dtype=np.int32), 0)
    assert gid.size == 0 and crank.size == 0 and ptr.tolist() == [0]


def test_bad_partition_rejected():
    sem, vert, E, N, glo, n_global = _setup()
    bad = np.zeros(E, dtype=np.int32)
    bad[3] = -1
    with pytest.raises(sem.SemError):
        sem.gs_halo(E, N, vert, bad, 0)
