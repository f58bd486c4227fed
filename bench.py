"""Benchmark of the SEM Poisson hot path on GB300.

Workload (default): synthetic O-grid straight pipe, R = 1, L = 8, nc = 16,
nr = 4, nzp = 512 -> E = 262,144 curved hexahedra at N = 7 (1.34e8 local GLL
points, 9.07e7 global nodes), RHS from a seeded smooth Gaussian-random
field.  One step = one complete Poisson solve to ||r|| <= 1e-10 ||b|| with the
mixed-precision refined Jacobi-PCG (FP32 inner CG, FP64 outer residual),
inputs resident in HBM.  The mesh data (~20 GB) is far larger than L2, so no
L2 flush is needed between steps.

Also measured in the same run (outside the timed steps): FP64 and FP32 Ax
GDOF/s and their roofline fractions, gather-scatter, one plain FP64 PCG
solve of the same system, the end-to-end solve through host buffers, and the
CPU oracle on a bounded sample (``cpu_baseline``).

``--impl reference`` times the CPU oracle (the plain numpy FP64
implementation in oracle/) on a bounded sample of the same workload and
prints the same JSON line with "impl": "reference".
"""

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 Ax GDOF/s & %HBM roofline; mixed-prec PCG solves/s, p50/p99 at 1e-10"
WORKLOAD = "pipe262144_n7"
# algorithmic bytes per local point (one read of u, G (6 factors), one write of w)
AX_BYTES = {"fp64": 64, "fp32": 32}
# Nominal dense FP64 rate of one GB300 on its CUDA cores, TFLOP/s.
FP64_NOMINAL_TFLOPS = 1.25


def ax_fp64_roofs(N, n_local, ms, hbm_gbs):
    """Both roofs of the FP64 Poisson operator of Alg. 1 and which one binds a
    kernel that evaluates it on the FP64 pipe: HBM at 64 B a local point, and
    FP64 arithmetic at 12 n + 18 flops a point (n = N + 1: three forward and
    three transposed derivative contractions of about 2 n flops each, the
    symmetric G applied to the gradient, 15, and the accumulation of the three
    transposed terms, 3).  `vs_binding_roof` is the binding roof's time over
    the measured time: above 1, the kernel beats what a native FP64 kernel
    could reach."""
    n = N + 1
    flops = 12 * n + 18
    hbm_ms = AX_BYTES["fp64"] * n_local / (hbm_gbs * 1e6)
    fp64_ms = flops * n_local / (FP64_NOMINAL_TFLOPS * 1e9)
    return {"flops_per_point": flops, "hbm_roof_ms": hbm_ms, "fp64_roof_ms": fp64_ms,
            "fp64_tflops_nominal": FP64_NOMINAL_TFLOPS, "binds": "fp64" if fp64_ms > hbm_ms else "hbm",
            "vs_binding_roof": max(hbm_ms, fp64_ms) / ms}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def pct(vals, q):
    v = sorted(vals)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def time_kernel(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def aggregate(local_seconds, steps, world, dist=None):
    """Whole-job throughput of N independent replicas: every rank solved
    `steps` systems in `local_seconds`; the job time is the maximum over
    ranks (one all-reduce; the data path has no collective)."""
    t = float(local_seconds)
    if world > 1 and dist is not None:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        tt = torch.tensor([t], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt)
    return world * steps / t, t


# ---------------------------------------------------------------- oracle arm

def _oracle_slab_worker(budget_s, warmup=0, steps=1):
    """One host core: the oracle's FP64 Jacobi-PCG iteration (A = mask QQ^T
    A_L, Jacobi, weighted dots; oracle/solver.py restated as a loop) on a
    3-layer slab of the bench pipe (nc = 16, nr = 4, N = 7, E = 1536):
    `warmup` untimed steps, then `steps` timed ones, each iterating for
    budget_s / steps seconds.  Returns (local points x iterations per second
    of each timed step, iterations, seconds)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import numpy as np
    from oracle import mesh as omesh, solver as osolver
    from sem_inputs import forcing
    m = omesh.pipe(16, 4, 3, 7, R=1.0, L=8.0 * 3 / 512, periodic=True)
    P = osolver.Problem(m)
    b = P.rhs(forcing.evaluate(m.xyz, forcing.random_modes(2, L=8.0)))
    Minv = P.jacobi_inverse()
    x = np.zeros(P.shape)
    r = b.copy()
    z = Minv * r
    p = z.copy()
    rho = P.dot(r, z)

    def run(seconds):
        nonlocal x, r, z, p, rho
        t0 = time.perf_counter()
        k = 0
        while True:
            w = P.A(p)
            alpha = rho / P.dot(p, w)
            x += alpha * p
            r -= alpha * w
            P.dot(r, r)
            z = Minv * r
            rho_new = P.dot(r, z)
            p = z + (rho_new / rho) * p
            rho = rho_new
            k += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                return k, el

    per_step = budget_s / max(1, steps)
    for _ in range(warmup):
        run(per_step)
    rates, its, secs = [], 0, 0.0
    for _ in range(max(1, steps)):
        k, el = run(per_step)
        rates.append(k * m.E * 512 / el)
        its += k
        secs += el
    return rates, its, secs


def _oracle_full_solve(workload):
    """One complete FP64 Jacobi-PCG solve by the oracle on the host (one
    core): the small configurations it can finish, with their own iteration
    counts.  Returns (iterations, seconds, relative residual)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import mesh as omesh, solver as osolver
    from sem_inputs import configs, forcing
    d = configs.mesh_desc(workload)
    if d["kind"] == "box":
        m = omesh.box(d["nx"], d["ny"], d["nz"], d["N"], d["lx"], d["ly"], d["lz"])
        f = forcing.manufactured(m.xyz)
    else:
        m = omesh.pipe(d["nc"], d["nr"], d["nzp"], d["N"], R=d["R"], L=d["L"], a=d["a"], beta=d["beta"], periodic=True)
        f = forcing.evaluate(m.xyz, forcing.random_modes(2, L=d["L"]))
    P = osolver.Problem(m)
    b = P.rhs(f)
    t0 = time.perf_counter()
    res = osolver.pcg(P, b, tol=1e-10)
    return res.iters, time.perf_counter() - t0, float(res.rel_res)


def start_oracle_full_solves(workloads=("box4_n7", "pipe4096_n7")):
    """The oracle's full solves of the small configurations, in spawned
    processes started before the GPU legs (they run alongside them)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(len(workloads))
    return pool, {w: pool.apply_async(_oracle_full_solve, (w,)) for w in workloads}


def collect_oracle_full_solves(handle, timeout_s=120.0):
    pool, jobs = handle
    out = {}
    t_end = time.perf_counter() + timeout_s
    for w, job in jobs.items():
        try:
            it, sec, rel = job.get(timeout=max(1.0, t_end - time.perf_counter()))
            out[w] = {"iters": it, "seconds": sec, "solves_per_s": 1.0 / sec, "rel_res": rel, "cores": 1}
        except Exception as e:  # not finished within the bench's time: reported, not waited for
            out[w] = {"error": f"{type(e).__name__}: not finished within the bench run"}
    pool.terminate()
    return out


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def oracle_sample(budget_s=20.0, cores=None, warmup=0, steps=1):
    """The oracle's FP64 PCG iteration timed on every host core at once: one
    spawned process per core, each iterating on its own copy of the 3-layer
    slab (independent problems, as the GPU replicas), `warmup` untimed and
    `steps` timed steps of budget_s / steps seconds each.  Returns (seconds
    per local point per iteration for the whole host, averaged over the timed
    steps, cores, CPU model, description, the same per timed step)."""
    import multiprocessing as mp
    ncores, model = host_cpu()
    cores = cores or ncores
    ctx = mp.get_context("spawn")  # no fork after CUDA initialisation
    with ctx.Pool(cores) as pool:
        res = pool.starmap(_oracle_slab_worker, [(budget_s, warmup, steps)] * cores)
    nsteps = len(res[0][0])
    step_rates = [sum(r[0][j] for r in res) for j in range(nsteps)]  # the host's rate in each step
    rate = sum(step_rates) / nsteps
    its = sum(r[1] for r in res)
    desc = (f"oracle FP64 Jacobi-PCG iterations on a 3-layer slab of the pipe (nc=16, nr=4, N=7, E=1536), one "
            f"process per core on {cores} cores ({model}), {budget_s:.0f} s each"
            + (f" in {nsteps} timed steps after {warmup} untimed" if nsteps > 1 or warmup else "")
            + f", {its} iterations in total; the host's points x iterations per second scaled to the solve")
    return 1.0 / rate, cores, model, desc, [1.0 / q for q in step_rates]


# FP64 Jacobi-PCG iterations of the bench system (E = 262,144 pipe, seed-2
# right-hand side, tol 1e-10), measured by the FP64 solve of this build on
# GB300 (its iteration counts are held to within 2 of the oracle's by the
# parity tests on smaller meshes).  The oracle cannot run a solve of this size
# on the host; the reference arm multiplies its measured per-iteration rate by
# this count.  The GPU arm uses the count its own FP64 solve measures in the
# same run.
FP64_ITERS_BENCH = 5564


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    E, n3 = 262144, 512
    # W untimed and K timed steps, each a bounded sample of the workload
    # (about 20 s of timed work in all, at least 2 s a step)
    budget = max(20.0, 2.0 * max(1, args.steps))
    sec_pt, cores, model, desc, step_sec_pt = oracle_sample(budget_s=budget, warmup=args.warmup, steps=args.steps)
    sec_per_solve = sec_pt * E * n3 * FP64_ITERS_BENCH
    value = 1.0 / sec_per_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_solve * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{WORKLOAD}: O-grid pipe E=262144 N=7, FP64 Jacobi-PCG to 1e-10"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "cpu": model, "kind": "oracle",
                             "sample": desc + f" and {FP64_ITERS_BENCH} iterations (the system's FP64 PCG count)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_values": [1.0 / (q * E * n3 * FP64_ITERS_BENCH) for q in step_sec_pt]}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- serving leg

def serving_stream(count, rate, seed=4, log2_e=(9.0, 15.0)):
    """Request stream through the batching server: Poisson arrivals at `rate`
    per second (rate = inf: all at once, which measures the saturation
    throughput); box or pipe meshes with E log-uniform in [512, 32768]; N in
    {5, 7, 9}; Poisson or Helmholtz (h2 log-uniform in [1e-2, 1e2]); mixed
    precision to 1e-10.  Latency = submit -> result visible to poll, with the
    server's breakdown of each request (queue, mesh set-up, wait for a batch
    slot, solve; sem_server_poll_timed)."""
    import numpy as np
    import paper_2109_03592_gb300 as sem
    from sem_inputs import serving
    stream = serving.request_stream(seed=seed, count=count, rate=rate if math.isfinite(rate) else 1.0,
                                    log2_e=log2_e)
    srv = sem.Server(max_slots=8)
    pending = {}
    t0 = time.perf_counter()
    for req in stream:
        if math.isfinite(rate):
            now = time.perf_counter() - t0
            if req["arrival"] > now:
                time.sleep(req["arrival"] - now)
        d = req["desc"]
        n = d["N"] + 1
        E = d["nx"] * d["ny"] * d["nz"] if d["kind"] == "box" else d["nc"] * (d["nc"] + 4 * d["nr"]) * d["nzp"]
        f = np.random.default_rng(req["seed"]).standard_normal(E * n ** 3)
        rid = srv.submit(d, f, tol=1e-10, h1=1.0, h2=req["h2"], prec=sem.MIXED)
        pending[rid] = E * n ** 3
    submit_s = time.perf_counter() - t0
    lat, worst, phases = [], 0.0, {"queue_ms": [], "setup_ms": [], "wait_ms": [], "solve_ms": []}
    for rid in pending:
        st, x, res = srv.poll(rid, timeout_ms=-1, timing=True)
        if st != sem.SEM_OK:
            raise RuntimeError(f"serving request failed: {st} {res}")
        tm = res["timing"]
        lat.append(tm["total_ms"])
        for k in phases:
            phases[k].append(tm[k])
        worst = max(worst, res["rel_res"])
    wall = time.perf_counter() - t0
    srv.close()
    return {"requests": count, "arrival_rate_per_s": rate if math.isfinite(rate) else "all at once",
            "offered_rate_per_s": count / submit_s if submit_s > 0 else None,
            "throughput_solves_per_s": count / wall,
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat)},
            "breakdown_ms_p50": {k: pct(v, 50) for k, v in phases.items()},
            "breakdown_ms_p99": {k: pct(v, 99) for k, v in phases.items()},
            "max_rel_res": worst, "mode": "batched per order (one CUDA graph per order per step)",
            "mix": (f"box/pipe, E log-uniform in [{2 ** log2_e[0]:.0f}, {2 ** log2_e[1]:.0f}], N in {{5,7,9}}, "
                    "Poisson/Helmholtz, tol 1e-10")}


def serving_sweep(count, seed=4):
    """The serving configuration's rate sweep: the saturation throughput from
    a burst of `count` requests, then Poisson streams of `count` requests at
    0.5x, 1x and 2x that rate."""
    sat = serving_stream(count, float("inf"), seed=seed)
    lam = sat["throughput_solves_per_s"]
    out = {"saturation": sat, "rates": []}
    for k, mult in enumerate((0.5, 1.0, 2.0)):
        out["rates"].append(dict(serving_stream(count, mult * lam, seed=seed + 1 + k), rate_over_saturation=mult))
    return out


# ---------------------------------------------------------------- projection leg

def projection_leg(count=6, max_vectors=8, workload="pipe32768_n7"):
    """Successive solves with slowly varying right-hand sides (as over time
    steps): the 64-mode random field with every phase advancing at its own
    rate, f_j = sum_m a_m cos(k_m x + phi_m + w_m t_j), w_m ~ U[0.5, 1.5],
    t_j = 0.05 j (the right-hand sides leave any finite span); mixed precision
    to 1e-10, with and without the projection space of earlier solutions
    (sem_proj_*)."""
    import numpy as np
    import torch
    import paper_2109_03592_gb300 as sem
    from sem_inputs import configs, forcing
    desc = configs.mesh_desc(workload)
    m = sem.Mesh(desc)
    xyz = m.coords()
    a, k, phi = forcing.random_modes(5, L=desc.get("L", 8.0))
    w = np.random.default_rng(7).uniform(0.5, 1.5, a.size)
    proj = sem.Projection(m, max_vectors=max_vectors)
    b = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    out = {"with": {"iters": [], "ms": []}, "without": {"iters": [], "ms": []}}
    for j in range(count):
        m.rhs(forcing.evaluate_torch(xyz, (a, k, phi + w * 0.05 * j)), b)
        r = proj.solve(b, x, tol=1e-10, prec=sem.MIXED)
        if r["status"] != 0:
            raise RuntimeError(f"projected solve failed: {r}")
        out["with"]["iters"].append(r["iters"])
        out["with"]["ms"].append(r["ms"])
        x.zero_()
        r = m.solve(b, x, tol=1e-10, prec=sem.MIXED)
        out["without"]["iters"].append(r["iters"])
        out["without"]["ms"].append(r["ms"])
    del xyz
    proj.close()
    m.close()
    tw, to = sum(out["with"]["ms"]), sum(out["without"]["ms"])
    return {"workload": f"{workload}: E={desc_elements(desc)} N={desc['N']}", "solves": count,
            "max_vectors": max_vectors, **out, "time_ratio": tw / to if to > 0 else None,
            "note": "first solve has an empty space; ms includes projection and basis update"}


def velocity_helmholtz_leg(workload, re=1.0e4, dt=2.0e-4, reps=5):
    """The velocity step of Sec. 2, Eq. 4: (b0/dt) u - div(nu grad u) / Re = rhs for the three
    velocity components on one mesh.  Per-point viscosity nu(x) (sem_mesh_set_coefficients,
    seeded smooth field times per-element jumps), h1 = 1/Re with Re = 1e4, h2 = b0/dt with BDF2's
    b0 = 3/2 and dt = 2e-4; mixed precision to 1e-10; the three solves as one batch
    (sem_pcg_solve_batch) and one at a time, the median of `reps` timings each."""
    import torch
    import paper_2109_03592_gb300 as sem
    from sem_inputs import coefficients, configs, forcing
    desc = configs.mesh_desc(workload)
    m = sem.Mesh(desc)
    xyz = m.coords()
    m.set_coefficients(torch.from_numpy(coefficients.viscosity(31, xyz.cpu().numpy())).cuda(), None)
    h1, h2 = 1.0 / re, 1.5 / dt
    bs = []
    for c in range(3):
        b = torch.empty(m.shape, dtype=torch.float64, device="cuda")
        m.rhs(forcing.evaluate_torch(xyz, forcing.random_modes(40 + c, L=desc.get("L", 8.0))), b)
        bs.append(b)
    del xyz
    opts = dict(tol=1e-10, h1=h1, h2=h2, prec=sem.MIXED)
    xs = [torch.zeros_like(b) for b in bs]

    def one_at_a_time():
        res = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, x in zip(bs, xs):
            x.zero_()
            res.append(m.solve(b, x, **opts))
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    def batched():
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res = sem.solve_batch([m] * 3, bs, xs, [dict(tol=1e-10, h1=h1, h2=h2)] * 3)
        torch.cuda.synchronize()
        if st != sem.SEM_OK:
            raise RuntimeError(f"velocity batch failed: {st} {res}")
        return res, time.perf_counter() - t0

    one_at_a_time()  # warm-up (graphs, workspaces, batch engine)
    batched()
    t_seq, t_bat = [], []
    for _ in range(reps):
        seq, t = one_at_a_time()
        t_seq.append(t)
        bat, t = batched()
        t_bat.append(t)
    t_seq, t_bat = sorted(t_seq)[reps // 2], sorted(t_bat)[reps // 2]
    m.close()
    for r in seq + bat:
        if r["status"] != 0:
            raise RuntimeError(f"velocity solve failed: {r}")
    return {"workload": f"{workload}: E={desc_elements(desc)} N={desc['N']}", "components": 3,
            "coefficients": "h1 = nu(x)/Re per point, Re = 1e4; h2 = b0/dt = 7500", "tol": 1e-10,
            "iters": [r["iters"] for r in bat], "iters_one_at_a_time": [r["iters"] for r in seq],
            "max_rel_res": max(r["rel_res"] for r in seq + bat),
            "batched_ms": t_bat * 1e3, "one_at_a_time_ms": t_seq * 1e3,
            "note": "median wall time of the three solves (host-synchronous calls, device-resident data)"}


def pressure_leg(m, stream, reps):
    """The consistent Poisson operator E = D B^-1 D^T of the P_N - P_{N-2}
    pressure space (Sec. 2, Eq. 5) on the bench mesh: sem_pressure_apply
    (weak gradient, three QQ^T with mask, inverse mass and weak divergence),
    timed with CUDA events on the launching stream after a first call that
    builds the GL-point factors.  Algorithmic work per element, m = N - 1 GL
    and n = N + 1 GLL points per direction: bytes = m^3 (p 8 + F 72 read twice
    + q 8) + n^3 (velocity 24 written and read, inverse mass 8) plus three
    FP64 QQ^T passes (20 B per shared point); FP64 multiply-adds = 9 (m (m^2 n
    + m n^2 + n^3)) for D^T and 9 (n (n^2 m + n m^2 + m^3)) for D."""
    import torch
    mm, n = m.N - 1, m.N + 1
    m3, n3 = mm ** 3, n ** 3
    p = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda")
    q = torch.empty_like(p)
    work = torch.empty(3 * m.n_local, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    m.pressure_apply(p, q, work)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    apply_ms = time_kernel(lambda: m.pressure_apply(p, q, work), reps, stream)
    p32, q32, work32 = p.float(), q.float(), work.float()
    m.pressure_apply_f32(p32, q32, work32)
    apply32_ms = time_kernel(lambda: m.pressure_apply_f32(p32, q32, work32), reps, stream)
    del p32, q32, work32
    u = work.view((3,) + m.shape)
    grad_ms = time_kernel(lambda: m.pressure_grad(p, u), reps, stream)
    div_ms = time_kernel(lambda: m.pressure_div(u, q), reps, stream)
    shared = 1.0 - (max(m.N - 1, 0) ** 3) / n3
    bytes_el = m3 * (8 + 2 * 72 + 8) + n3 * (2 * 24 + 8) + 3 * 20 * shared * n3
    fma_el = 9 * (mm * (mm * mm * n + mm * n * n + n3)) + 9 * (n * (n * n * mm + n * mm * mm + m3))
    dofs = m.E * m3
    del p, q, work, u
    return {"workload": f"E={m.E} N={m.N}: {dofs} pressure values on the GL points",
            "apply_ms": apply_ms, "apply_fp32_ms": apply32_ms, "grad_ms": grad_ms, "div_ms": div_ms,
            "first_call_ms": setup_ms,
            "gdofs": dofs / (apply_ms * 1e6),
            "algorithmic_gbs": bytes_el * m.E / (apply_ms * 1e6),
            "fp64_tflops": 2 * fma_el * m.E / (apply_ms * 1e9),
            "bound": "fp64 pipe (native FP64 contractions)"}


def pressure_solve_leg(workload="pipe4096_n7", tol=1e-10):
    """Solves of the pressure equation E p = g (Sec. 2, Eq. 5) on the
    mean-free space (sem_pressure_solve, CG) on the E = 4096 pipe, the paper's
    per-GPU regime, g a seeded standard-normal pressure field: FP64, and mixed
    precision (FP32 E, FP64 reliable updates), both Jacobi-preconditioned
    (diag(E)), and the plain FP64 CG beside them.  The first operator calls
    (which build the GL-point factors, their FP32 copies and the diagonal)
    are made before timing."""
    import torch
    import paper_2109_03592_gb300 as sem
    from sem_inputs import configs
    m = sem.Mesh(configs.mesh_desc(workload))
    g = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(4))
    x = torch.empty_like(g)
    m.pressure_apply(g, x)
    m.pressure_apply_f32(g.float(), x.float())
    m.pressure_solve(g, x, tol=tol, maxit=1)  # builds diag(E)
    torch.cuda.synchronize()
    r = m.pressure_solve(g, x, tol=tol)
    out = {"workload": f"{workload}: E={m.E} N={m.N}, {m.pressure_size()} pressure values", "tol": tol,
           "iters": r["iters"], "ms": r["ms"], "ms_per_iter": r["ms"] / max(1, r["iters"]),
           "rel_res": r["rel_res"], "status": r["status"]}
    rm = m.pressure_solve(g, x, tol=tol, prec=sem.MIXED)
    out["mixed"] = {"iters": rm["iters"], "replacements": rm["outer_iters"], "ms": rm["ms"], "rel_res": rm["rel_res"],
                    "status": rm["status"]}
    rp = m.pressure_solve(g, x, tol=tol, precond=sem.PRECOND_NONE)
    out["unpreconditioned"] = {"iters": rp["iters"], "ms": rp["ms"], "rel_res": rp["rel_res"], "status": rp["status"]}
    m.close()
    return out


def _sig(obj, digits=4):
    """Floats rounded to `digits` significant digits (auxiliary legs only)."""
    if isinstance(obj, float):
        return float(f"{obj:.{digits}g}") if math.isfinite(obj) else obj
    if isinstance(obj, dict):
        return {k: _sig(v, digits) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [_sig(v, digits) for v in obj]
    return obj


def compact_projection(p):
    if not p:
        return p
    return _sig({"workload": p["workload"], "solves": p["solves"], "iters_with": p["with"]["iters"],
                 "iters_without": p["without"]["iters"], "ms_with": sum(p["with"]["ms"]),
                 "ms_without": sum(p["without"]["ms"]), "time_ratio": p["time_ratio"]})


def compact_velocity(v):
    if not v:
        return v
    return [_sig({"workload": r["workload"], "iters": r["iters"], "batched_ms": r["batched_ms"],
                  "one_at_a_time_ms": r["one_at_a_time_ms"], "max_rel_res": r["max_rel_res"]}) for r in v]


def compact_pressure(p):
    if not p or "error" in p:
        return p
    out = {k: p[k] for k in ("apply_ms", "apply_fp32_ms", "grad_ms", "div_ms", "gdofs", "fp64_tflops",
                             "algorithmic_gbs") if k in p}
    if "solve" in p:
        sv = p["solve"]
        out["solve"] = sv if "error" in sv else {k: sv[k] for k in ("iters", "ms", "rel_res", "status", "mixed",
                                                                       "unpreconditioned")
                                                  if k in sv}
    return _sig(out)


def schwarz_leg(m, b, stream, precs=("MIXED",)):
    """The overlapping Schwarz preconditioner (Sec. 2, Eq. 6; sem_schwarz_*)
    on the bench system: set-up, one application (FP32 and FP64, CUDA events
    on the launching stream) and solves to 1e-10 beside the Jacobi ones."""
    import torch
    import paper_2109_03592_gb300 as sem
    t0 = time.perf_counter()
    sw = sem.Schwarz(m, coarse=True)
    setup_s = time.perf_counter() - t0
    info = sw.info()
    out = {"setup_s": setup_s, "coarse": info["coarse"], "n_coarse": info["n_coarse"],
           "n_distinct_1d": info["n_distinct"]}
    r32 = torch.randn(m.shape, dtype=torch.float32, device="cuda")
    m.gs(r32, apply_mask=True, prec=sem.FP32)
    z32 = torch.empty_like(r32)
    out["apply_fp32_ms"] = time_kernel(lambda: sw.apply(r32, z32, prec=sem.FP32), 5, stream)
    del r32, z32
    x = torch.zeros_like(b)
    for prec in precs:
        x.zero_()
        r = sw.solve(b, x, tol=1e-10, prec=getattr(sem, prec))
        out[prec.lower()] = {"iters": r["iters"], "ms": r["ms"], "solves_per_s": 1e3 / r["ms"],
                             "rel_res": r["rel_res"], "status": r["status"]}
    sw.close()
    return _sig(out)


def large_leg(workloads=("pipe1048576_n7", "pipe131072_n11"), precs=("MIXED",)):
    """The large configurations (E = 1,048,576 at N = 7, ~3.6e8 DOFs; E =
    131,072 at N = 11): mesh set-up, Jacobi-PCG solves to 1e-10 (time,
    iterations, the solver's true residual; mixed precision by default, FP64
    too with --large-fp64, ~4 more minutes) and the device memory in use
    during the solves (cudaMemGetInfo)."""
    import torch
    import paper_2109_03592_gb300 as sem
    from sem_inputs import configs, forcing
    out = []
    for wl in workloads:
        desc = configs.mesh_desc(wl)
        t0 = time.perf_counter()
        mm = sem.Mesh(desc)
        setup_s = time.perf_counter() - t0
        xyz = mm.coords()
        f = forcing.evaluate_torch(xyz, forcing.random_modes(2, L=desc.get("L", 8.0)))
        del xyz
        bb = torch.empty_like(f)
        mm.rhs(f, bb)
        del f
        torch.cuda.empty_cache()
        rec = {"workload": wl, "E": mm.E, "N": mm.N, "dofs": mm.E * mm.N ** 3, "setup_s": setup_s}
        xx = torch.zeros_like(bb)
        for prec in precs:
            xx.zero_()
            r = mm.solve(bb, xx, tol=1e-10, prec=getattr(sem, prec))
            free, total = torch.cuda.mem_get_info()
            rec[prec.lower()] = {"ms": r["ms"], "iters": r["iters"], "rel_res": r["rel_res"], "status": r["status"],
                                 "device_used_gb": (total - free) / 1e9}
        mm.close()
        del bb, xx
        torch.cuda.empty_cache()
        out.append(_sig(rec))
    return out


def desc_elements(d):
    return d["nx"] * d["ny"] * d["nz"] if d["kind"] == "box" else d["nc"] * (d["nc"] + 4 * d["nr"]) * d["nzp"]


# ---------------------------------------------------------------- GPU arm

# DRAM bytes (read + write) of one launch of the plain FP32 bulk-copy kernel
# tma::k_ax_tma<7, 2, 3, false>, from ncu on the E = 32,768 pipe (N = 7):
# 469,796,096 + 55,301,888 bytes.  The kernel streams its elements once
# (no reuse across elements), so a launch over E elements moves E / 32,768
# times that (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on one
# launch of this script with --workload pipe32768_n7).
TRAFFIC_E32768_N7 = 469_796_096 + 55_301_888
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of tma::k_ax_tma<7, 2, 3, false> on the "
                  "E = 32,768 pipe, scaled by the element count")


def fp32_ax_traffic(m):
    import paper_2109_03592_gb300 as sem
    if m.N != 7 or m.ax_variant(sem.FP32) != 2:  # the FP32 requests must run the measured kernel
        return None
    return TRAFFIC_E32768_N7 * m.E / 32768


def fp32_kernel_name(N, variant):
    """The FP32 local-operator kernel the autotuner chose (variants 0/1:
    register kernels with ~256/~128 threads per CTA; 2/3: persistent
    bulk-copy pipelined kernels with 3/2 stages)."""
    n2 = (N + 1) ** 2
    epb = max(1, (256 if variant in (0, 3) else 128) // n2)
    if variant >= 2:
        return f"tma::k_ax_tma<{N}, {epb}, {3 if variant == 2 else 2}, false> (FP32 local operator, bulk-copy pipelined)"
    return f"k_ax<{N}, float, {epb}, false> (FP32 local operator)"



def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2109_03592_gb300 as sem
    from sem_inputs import configs, forcing

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    full_cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        full_cpu = start_oracle_full_solves()
    desc = configs.mesh_desc(args.workload)
    t0 = time.perf_counter()
    m = sem.Mesh(desc)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    xyz = m.coords()
    f = forcing.evaluate_torch(xyz, forcing.random_modes(2 + rank, L=desc.get("L", 8.0)))
    del xyz
    b = torch.empty_like(f)
    m.rhs(f, b)
    del f
    x = torch.zeros_like(b)
    opts = dict(tol=1e-10, prec=sem.MIXED)

    for _ in range(args.warmup):
        x.zero_()
        m.solve(b, x, **opts)
    torch.cuda.synchronize()

    # ---- timed steps: K mixed-precision solves
    lat, iters, outers, rel = [], [], [], []
    launches0 = sem.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        dev_ms = 0.0
        for _ in range(args.steps):
            x.zero_()
            r = m.solve(b, x, **opts)
            lat.append(r["ms"])
            dev_ms += r["ms"]
            iters.append(r["iters"])
            outers.append(r["outer_iters"])
            rel.append(r["rel_res"])
            if r["status"] != 0:
                raise RuntimeError(f"solve failed: {r}")
        torch.cuda.synchronize()
        barrier()
        wall_s = time.perf_counter() - t_start
    launches = sem.kernel_launches() - launches0
    value, t_max = aggregate(dev_ms / 1e3, args.steps, world, dist if world > 1 else None)

    # ---- kernel-level measurements (same mesh, same stream the kernels run on)
    P = m.n_local
    dof = m.E * m.N ** 3
    hbm, peak_kind = peaks()
    u64 = torch.randn(m.shape, dtype=torch.float64, device="cuda")
    w64 = torch.empty_like(u64)
    reps = 5 if args.quick else 10
    ax64_ms = time_kernel(lambda: m.ax(u64, w64), reps, stream)
    u32 = u64.float()
    w32 = torch.empty_like(u32)
    ax32_ms = time_kernel(lambda: m.ax(u32, w32, prec=sem.FP32), 2 * reps, stream)
    gs64_ms = time_kernel(lambda: m.gs(w64, apply_mask=True), reps, stream)
    gs32_ms = time_kernel(lambda: m.gs(w32, apply_mask=True, prec=sem.FP32), reps, stream)
    del u64, w64, u32, w32
    pressure = None
    if not args.no_pressure:
        try:
            pressure = pressure_leg(m, stream, reps)
        except Exception as e:  # an auxiliary leg must not cost the headline line
            pressure = {"error": f"{type(e).__name__}: {e}"}
    ax32_gbs = AX_BYTES["fp32"] * P / (ax32_ms * 1e6)
    ax64_gbs = AX_BYTES["fp64"] * P / (ax64_ms * 1e6)

    # ---- plain FP64 PCG on the same system (one solve), and the mixed
    # solution's error against it: ||x_mixed - x_fp64||_W / ||x_fp64||_W
    fp64 = None
    mixed_err = None
    if not args.quick:
        x_mixed = x.clone()
        x.zero_()
        r64 = m.solve(b, x, tol=1e-10, prec=sem.FP64)
        fp64 = {"ms": r64["ms"], "iters": r64["iters"], "rel_res": r64["rel_res"], "status": r64["status"]}
        mult, _ = m.weights()
        d = x_mixed - x
        mixed_err = float(torch.sqrt((d * d / mult).sum() / (x * x / mult).sum()))
        del x_mixed, d, mult

    # ---- end to end through host buffers (pinned), same metric
    b_host = torch.empty(m.shape, dtype=torch.float64, pin_memory=True)
    b_host.copy_(b)
    x_host = torch.zeros(m.shape, dtype=torch.float64, pin_memory=True)
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 2))):
        x_host.zero_()
        r = m.solve_host(b_host.numpy(), x_host.numpy(), **opts)
        e2e_ms.append(r["ms"])
    e2e_value = world * len(e2e_ms) / (sum(e2e_ms) / 1e3)

    serving = None
    if not args.no_serving:
        serving = (serving_sweep(args.serving_requests) if args.serving_sweep
                   else serving_stream(args.serving_requests, args.serving_rate))
    proj = None
    if not args.no_projection:
        proj = projection_leg()
    if pressure is not None and "error" not in pressure:
        try:
            pressure["solve"] = pressure_solve_leg()
        except Exception as e:
            pressure["solve"] = {"error": f"{type(e).__name__}: {e}"}
    velocity = None
    if not args.no_velocity:
        velocity = [velocity_helmholtz_leg(w) for w in ("pipe4096_n7", "pipe32768_n7")]
    schwarz_res = None
    if not args.no_schwarz:
        try:
            schwarz_res = schwarz_leg(m, b, stream)
        except Exception as e:  # an auxiliary leg must not cost the headline line
            schwarz_res = {"error": f"{type(e).__name__}: {e}"}
    mesh_E, mesh_N, mesh_glob = m.E, m.N, m.n_global
    fp32_var, fp64_df, ax_traffic = m.ax_variant(sem.FP32), m.fp64_double_float(), fp32_ax_traffic(m)
    large = None
    if not args.no_large:
        m.close()  # the large meshes need the device memory
        del b, x
        torch.cuda.empty_cache()
        try:
            large = large_leg(precs=("MIXED", "FP64") if args.large_fp64 else ("MIXED",))
        except Exception as e:
            large = {"error": f"{type(e).__name__}: {e}"}

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            sec_pt, cores, model, desc_s, _ = oracle_sample(budget_s=20.0)
            iters_cpu = fp64["iters"] if fp64 else FP64_ITERS_BENCH
            sec = sec_pt * P * iters_cpu
            cpu = {"value": 1.0 / sec, "unit": "solves/s", "cores": cores, "cpu": model, "kind": "oracle",
                   "sample": desc_s + f" and {iters_cpu} iterations (the FP64 PCG count of this system)"}
            if full_cpu is not None:
                cpu["full_solves"] = _sig(collect_oracle_full_solves(full_cpu))
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer (mixed, reliable updates)",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: O-grid pipe E={mesh_E} N={mesh_N}, mixed-precision Jacobi-PCG "
                                   f"to 1e-10 (FP32 inner, FP64 outer residual)",
                       "E": mesh_E, "N": mesh_N, "n_local": P, "n_global": mesh_glob, "tol": 1e-10,
                       "l2": "inputs larger than L2 (mesh ~20 GB), no flush", "replicas": world,
                       "setup_s": round(setup_s, 2)},
            "roofline": {"bound": "hbm", "kernel": fp32_kernel_name(mesh_N, fp32_var),
                         "timed": "sem_ax FP32 launches on the bench mesh, CUDA events on the launching stream, "
                                  "after the timed solves (the inner CG runs the fused form of the same kernel)",
                         "achieved": ax32_gbs, "peak": hbm, "unit": "GB/s", "frac": ax32_gbs / hbm,
                         "peak_kind": peak_kind, "traffic": ax_traffic,
                         "traffic_source": TRAFFIC_SOURCE,
                         "algorithmic_bytes_per_launch": AX_BYTES["fp32"] * P},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 2 * 8 * P,
                    "d2h_bytes_per_step": 8 * P, "ms": e2e_ms},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "min": min(lat), "max": max(lat)},
            "solve": {"iters": iters[0], "outer_iters": outers[0], "max_rel_res": max(rel), "wall_s": wall_s},
            # auxiliary legs, compact; the headline's secondary metrics come last
            "projection": compact_projection(proj),
            "velocity_helmholtz": compact_velocity(velocity),
            "pressure_operator": compact_pressure(pressure),
            "large": large,
            "serving": _sig(serving) if serving else serving,
            "schwarz": schwarz_res,
            "fp64_pcg": fp64,
            "mixed_vs_fp64_err": mixed_err,
            "gs": {"fp64_ms": gs64_ms, "fp32_ms": gs32_ms},
            "ax": {"fp64_ms": ax64_ms, "fp64_gdofs": dof / (ax64_ms * 1e6), "fp64_gbs": ax64_gbs,
                   "fp64_hbm_frac": ax64_gbs / hbm, "fp64_kernel": "double-float" if fp64_df else "native",
                   "fp64_roofs": ax_fp64_roofs(mesh_N, P, ax64_ms, hbm),
                   "fp32_ms": ax32_ms, "fp32_gdofs": dof / (ax32_ms * 1e6), "fp32_gbs": ax32_gbs,
                   "fp32_hbm_frac": ax32_gbs / hbm},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sem", choices=["sem", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--quick", action="store_true", help="skip the FP64 PCG comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-projection", action="store_true", help="skip the projection leg")
    ap.add_argument("--no-pressure", action="store_true", help="skip the P_N - P_{N-2} pressure-operator leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream leg")
    ap.add_argument("--no-velocity", action="store_true", help="skip the three-component velocity Helmholtz leg")
    ap.add_argument("--no-schwarz", action="store_true", help="skip the overlapping-Schwarz leg")
    ap.add_argument("--no-large", action="store_true", help="skip the E = 1,048,576 and N = 11 solves")
    ap.add_argument("--large-fp64", action="store_true", help="also the FP64 solves of the large configurations")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-rate", type=float, default=2.0)
    ap.add_argument("--serving-sweep", action="store_true",
                    help="saturation burst, then streams at 0.5x, 1x, 2x the saturation rate")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
