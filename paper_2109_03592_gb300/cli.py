"""Command-line solves on the synthetic workloads, for scripting and profiling.

    python -m paper_2109_03592_gb300.cli solve --workload pipe32768_n7 --prec fp64 [--repeat 2]
    python -m paper_2109_03592_gb300.cli ax --workload pipe262144_n7 --prec fp64 [--reps 10]
    python -m paper_2109_03592_gb300.cli gs --workload pipe262144_n7 --prec fp32 [--reps 10]
    python -m paper_2109_03592_gb300.cli ax --workload pipe262144_n7 --prec fp32 --coef
    python -m paper_2109_03592_gb300.cli pressure --workload pipe32768_n7 [--reps 10]
    python -m paper_2109_03592_gb300.cli psolve --workload pipe4096_n7 [--tol 1e-10] [--no-precond]
    python -m paper_2109_03592_gb300.cli schwarz --workload pipe262144_n7 --prec mixed [--no-coarse]

pressure times the consistent Poisson operator E = D B^-1 D^T of the
P_N - P_{N-2} pressure space (sem_pressure_apply; --prec fp32:
sem_pressure_apply_f32); psolve solves E p = g on the mean-free pressure
space (sem_pressure_solve, --prec fp64 or mixed) for a seeded
standard-normal g.

schwarz solves with the overlapping Schwarz preconditioner (sem_schwarz_*)
instead of Jacobi.

--coef gives the mesh seeded per-point coefficients h1(i,j,k,e), h2(i,j,k,e)
(a variable viscosity and mass coefficient) before the timed calls, which then
use h1 = h2 = 1.

Prints one JSON line per solve (the sem_pcg_solve result) or per operator /
gather-scatter timing (CUDA events on the launching stream).
"""

import argparse
import json
import sys


def _mesh_and_rhs(workload):
    import torch
    from sem_inputs import configs, forcing
    from . import sem
    desc = configs.mesh_desc(workload)
    m = sem.Mesh(desc)
    xyz = m.coords()
    f = forcing.evaluate_torch(xyz, forcing.random_modes(2, L=desc.get("L", 8.0)))
    del xyz
    b = torch.empty_like(f)
    m.rhs(f, b)
    return m, b


def _set_coefficients(m):
    import torch
    from sem_inputs import coefficients
    xyz = m.coords().cpu().numpy()
    h1 = torch.from_numpy(coefficients.viscosity(21, xyz)).cuda()
    h2 = torch.from_numpy(coefficients.mass_coefficient(22, xyz)).cuda()
    m.set_coefficients(h1, h2)


def _pressure(args):
    import torch
    from sem_inputs import configs
    from . import sem
    m = sem.Mesh(configs.mesh_desc(args.workload))
    g = torch.randn(m.pressure_shape, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(4))
    q = torch.empty_like(g)
    work = torch.empty(3 * m.n_local, dtype=torch.float64, device="cuda")
    if args.what == "psolve":
        m.pressure_apply(g, q, work)  # builds the GL-point factors
        prec = sem.MIXED if args.prec == "mixed" else sem.FP64
        precond = sem.PRECOND_NONE if args.no_precond else sem.PRECOND_JACOBI
        for _ in range(args.repeat):
            r = m.pressure_solve(g, q, tol=args.tol, prec=prec, precond=precond)
            print(json.dumps({"workload": args.workload, "prec": "mixed" if prec == sem.MIXED else "fp64",
                              "precond": "none" if args.no_precond else "jacobi",
                              "pressure_values": m.pressure_size(), **r}), flush=True)
    else:
        f32 = args.prec == "fp32"
        if f32:
            g, q = g.float(), q.float()
            work = work.float()
        apply = (lambda: m.pressure_apply_f32(g, q, work)) if f32 else (lambda: m.pressure_apply(g, q, work))
        for _ in range(3):
            apply()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.reps):
            apply()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / args.reps
        print(json.dumps({"workload": args.workload, "ms": ms, "pressure_values": m.pressure_size(),
                          "gdofs": m.pressure_size() / ms / 1e6}), flush=True)
    m.close()
    return 0


def main(argv=None):
    from . import sem
    ap = argparse.ArgumentParser(prog="python -m paper_2109_03592_gb300.cli")
    ap.add_argument("what", choices=["solve", "ax", "gs", "pressure", "psolve", "schwarz"])
    ap.add_argument("--workload", default="pipe32768_n7")
    ap.add_argument("--prec", default="mixed", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--coef", action="store_true", help="per-point h1, h2 on the mesh (h1 = h2 = 1 in the calls)")
    ap.add_argument("--helmholtz", action="store_true", help="h2 = 1 (the mass term) with scalar coefficients")
    ap.add_argument("--no-coarse", action="store_true", help="schwarz: local solves only")
    ap.add_argument("--no-precond", action="store_true", help="psolve: plain CG (default: Jacobi, diag(E))")
    args = ap.parse_args(argv)
    import torch
    prec = {"fp64": sem.FP64, "fp32": sem.FP32, "mixed": sem.MIXED}[args.prec]
    if args.what in ("pressure", "psolve"):
        return _pressure(args)
    m, b = _mesh_and_rhs(args.workload)
    h1, h2 = 1.0, 1.0 if args.helmholtz else 0.0
    if args.coef:
        _set_coefficients(m)
        h2 = 1.0
    if args.what == "schwarz":
        sw = sem.Schwarz(m, h1, h2, coarse=not args.no_coarse)
        x = torch.zeros_like(b)
        for _ in range(args.repeat):
            x.zero_()
            r = sw.solve(b, x, tol=args.tol, prec=prec, h1=h1, h2=h2)
            print(json.dumps({"workload": args.workload, "prec": args.prec, "preconditioner": "schwarz",
                              **sw.info(), **r}), flush=True)
        sw.close()
    elif args.what == "solve":
        x = torch.zeros_like(b)
        for _ in range(args.repeat):
            x.zero_()
            r = m.solve(b, x, tol=args.tol, prec=prec, h1=h1, h2=h2)
            print(json.dumps({"workload": args.workload, "prec": args.prec, "coef": args.coef, **r}), flush=True)
    elif args.what == "gs":
        dt = torch.float32 if prec == sem.FP32 else torch.float64
        p = sem.FP32 if prec == sem.FP32 else sem.FP64
        v = torch.randn(m.shape, dtype=dt, device="cuda")
        for _ in range(3):
            m.gs(v, apply_mask=True, prec=p)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.reps):
            m.gs(v, apply_mask=True, prec=p)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / args.reps
        esz = 4 if p == sem.FP32 else 8
        print(json.dumps({"workload": args.workload, "prec": args.prec, "ms": ms, "shared_points": m.n_seg_points,
                          "alg_gbs": m.n_seg_points * (4 + 2 * esz) / ms / 1e6}), flush=True)
    else:
        dt = torch.float32 if prec == sem.FP32 else torch.float64
        u = torch.randn(m.shape, dtype=dt, device="cuda")
        w = torch.empty_like(u)
        p = sem.FP32 if prec == sem.FP32 else sem.FP64
        for _ in range(3):
            m.ax(u, w, h1, h2, prec=p)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.reps):
            m.ax(u, w, h1, h2, prec=p)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / args.reps
        print(json.dumps({"workload": args.workload, "prec": args.prec, "coef": args.coef, "h2": h2, "ms": ms,
                          "gdofs": m.E * m.N ** 3 / ms / 1e6, "variant": m.ax_variant(p)}), flush=True)
    m.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
