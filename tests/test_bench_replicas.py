"""The multi-GPU form of bench.py is N independent replicas; its only
collective is the max-over-ranks job time.  Checked with two gloo ranks on
the CPU (no GPU involved)."""

import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, t = bench.aggregate(1.0 + rank, steps=3, world=world, dist=dist)
    out.put((rank, value, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_with_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    for rank, value, t in res:
        assert t == 2.0                      # max over ranks
        assert value == pytest.approx(3.0)   # 2 ranks x 3 solves / 2 s


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.aggregate(4.0, steps=2, world=1)
    assert t == 4.0 and value == 0.5


def test_fp64_operator_roofs():
    """E = 262,144, N = 7: 64 B and 114 flops a point; the FP64 pipe binds."""
    sys.path.insert(0, ROOT)
    import bench
    P = 262144 * 512
    r = bench.ax_fp64_roofs(7, P, 3.16, 6786.6)
    assert r["flops_per_point"] == 114
    assert r["binds"] == "fp64"
    assert r["hbm_roof_ms"] == pytest.approx(64 * P / 6786.6e6)
    assert r["fp64_roof_ms"] == pytest.approx(114 * P / 1.25e9)
    assert r["vs_binding_roof"] == pytest.approx(r["fp64_roof_ms"] / 3.16)
    assert bench.ax_fp64_roofs(1, 8, 1.0, 1e-9)["binds"] == "hbm"  # a slow memory


def test_oracle_sample_reports_each_timed_step():
    """The CPU oracle arm's sampler: two spawned processes, one untimed and
    two timed steps; the mean of the per-step values is the reported one."""
    sys.path.insert(0, ROOT)
    import bench
    sec_pt, cores, model, desc, steps = bench.oracle_sample(budget_s=1.0, cores=2, warmup=1, steps=2)
    assert cores == 2 and len(steps) == 2 and all(s > 0 for s in steps)
    rate = sum(1.0 / s for s in steps) / 2
    assert sec_pt == pytest.approx(1.0 / rate)
    assert "2 timed steps after 1 untimed" in desc
