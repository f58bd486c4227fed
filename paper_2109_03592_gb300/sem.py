"""Thin ctypes binding of the C ABI in include/sem.h (argument marshalling
only: every step of the hot path runs in libsem.so's CUDA kernels).

Device buffers are passed as torch CUDA tensors (their data_ptr()), host
buffers as numpy arrays.  There is no CPU fallback: if libsem.so is missing
or the GPU is unusable, the calls raise.
"""

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsem.so")

SEM_OK, SEM_ERR_INVALID, SEM_ERR_OOM, SEM_ERR_CUDA = 0, 1, 2, 3
SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN, SEM_ERR_BUSY, SEM_ERR_DEVICE_TIMEOUT = 4, 5, 6, 7
SEM_ERR_BAD_MESH, SEM_ERR_TIMEOUT, SEM_ERR_NOT_FOUND, SEM_ERR_CANCELLED = 8, 9, 10, 11
NOALLOC_MAX_POINTS = 1 << 18
FP64, FP32, MIXED = 0, 1, 2
PRECOND_DEFAULT, PRECOND_NONE, PRECOND_JACOBI = 0, 1, 2
KIND = {"box": 0, "pipe": 1, "explicit": 2}


class SemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("N", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("nc", C.c_int), ("nr", C.c_int), ("nzp", C.c_int),
                ("R", C.c_double), ("L", C.c_double), ("a", C.c_double), ("beta", C.c_double),
                ("periodic_z", C.c_int),
                ("E", C.c_int64), ("xyz", C.c_void_p), ("vert", C.c_void_p), ("dirichlet_face", C.c_void_p)]


class MeshInfo(C.Structure):
    _fields_ = [("E", C.c_int64), ("N", C.c_int), ("n_local", C.c_int64), ("n_global", C.c_int64),
                ("n_segments", C.c_int64), ("n_seg_points", C.c_int64), ("dev_bytes", C.c_size_t)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("h1", C.c_double), ("h2", C.c_double), ("inner_tol", C.c_double),
                ("maxit", C.c_int), ("max_outer", C.c_int), ("prec", C.c_int), ("refine", C.c_int),
                ("delta", C.c_double), ("precond", C.c_int)]


class SolveResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("rel_res", C.c_double), ("ms", C.c_double),
                ("status", C.c_int)]

    def as_dict(self):
        return dict(iters=self.iters, outer_iters=self.outer_iters, rel_res=self.rel_res, ms=self.ms,
                    status=self.status)


class SchwarzInfo(C.Structure):
    _fields_ = [("n_distinct", C.c_int64), ("n_coarse", C.c_int64), ("coarse", C.c_int), ("dev_bytes", C.c_size_t),
                ("setup_ms", C.c_double)]


class RequestTiming(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("setup_ms", C.c_double), ("wait_ms", C.c_double),
                ("solve_ms", C.c_double), ("total_ms", C.c_double)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("max_queue", C.c_int),
                ("device", C.c_int), ("batch", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("cancelled", C.c_uint64), ("queued", C.c_int), ("running", C.c_int),
                ("hbm_in_use", C.c_size_t), ("hbm_budget", C.c_size_t)]


# name -> (restype, argtypes); every entry point declared in include/sem.h
_P = C.c_void_p
SIGNATURES = {
    "sem_mesh_create": (C.c_int, [C.POINTER(MeshDesc), _P, C.POINTER(_P)]),
    "sem_mesh_destroy": (C.c_int, [_P]),
    "sem_mesh_info": (C.c_int, [_P, C.POINTER(MeshInfo)]),
    "sem_mesh_global_ids": (C.c_int, [_P, _P]),
    "sem_mesh_coords": (C.c_int, [_P, _P, _P]),
    "sem_mesh_geometry": (C.c_int, [_P, _P, _P, _P]),
    "sem_mesh_set_coefficients": (C.c_int, [_P, _P, _P, _P]),
    "sem_mesh_weights": (C.c_int, [_P, _P, _P, _P]),
    "sem_ax": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.c_int, _P]),
    "sem_gs": (C.c_int, [_P, _P, C.c_int, C.c_int, _P]),
    "sem_rhs": (C.c_int, [_P, _P, _P, _P]),
    "sem_apply": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P]),
    "sem_jacobi": (C.c_int, [_P, C.c_double, C.c_double, _P, _P]),
    "sem_pcg_solve": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "sem_proj_create": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.POINTER(_P)]),
    "sem_proj_destroy": (C.c_int, [_P]),
    "sem_proj_solve": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "sem_proj_size": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "sem_proj_reset": (C.c_int, [_P]),
    "sem_pcg_solve_host": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "sem_pcg_solve_noalloc": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "sem_pcg_solve_batch": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), C.c_int, _P]),
    "sem_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(_P)]),
    "sem_server_submit": (C.c_int, [_P, C.POINTER(MeshDesc), _P, C.POINTER(SolveOpts), C.POINTER(C.c_uint64)]),
    "sem_server_poll": (C.c_int, [_P, C.c_uint64, C.c_int, _P, C.POINTER(SolveResult)]),
    "sem_server_poll_timed": (C.c_int, [_P, C.c_uint64, C.c_int, _P, C.POINTER(SolveResult),
                                        C.POINTER(RequestTiming)]),
    "sem_server_cancel": (C.c_int, [_P, C.c_uint64]),
    "sem_server_stats_get": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "sem_server_destroy": (C.c_int, [_P]),
    "sem_topology_numbering": (C.c_int, [C.c_int64, C.c_int, _P, _P, C.POINTER(C.c_int64)]),
    "sem_gs_halo": (C.c_int, [C.c_int64, C.c_int, _P, _P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              _P, _P, _P, _P]),
    "sem_mesh_vertices": (C.c_int, [C.POINTER(MeshDesc), _P, C.POINTER(C.c_int64)]),
    "sem_status_str": (C.c_char_p, [C.c_int]),
    "sem_last_error": (C.c_char_p, []),
    "sem_version": (C.c_int, []),
    "sem_kernel_launches": (C.c_uint64, []),
    "sem_mesh_fp64_kernel": (C.c_int, [_P]),
    "sem_mesh_check": (C.c_int, [_P, _P]),
    "sem_mesh_ax_variant": (C.c_int, [_P, C.c_int]),
    "sem_pressure_basis": (C.c_int, [C.c_int, _P, _P, _P, _P]),
    "sem_schwarz_fdm_1d": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _P, _P]),
    "sem_schwarz_setup_host": (C.c_int, [C.c_int64, C.c_int, _P, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "sem_schwarz_create": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.POINTER(_P)]),
    "sem_schwarz_destroy": (C.c_int, [_P]),
    "sem_schwarz_info": (C.c_int, [_P, C.POINTER(SchwarzInfo)]),
    "sem_schwarz_apply": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "sem_schwarz_solve": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "sem_pressure_info": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "sem_pressure_diag": (C.c_int, [_P, _P, _P]),
    "sem_pressure_factors": (C.c_int, [_P, _P, _P]),
    "sem_pressure_grad": (C.c_int, [_P, _P, _P, _P]),
    "sem_pressure_div": (C.c_int, [_P, _P, _P, _P]),
    "sem_pressure_apply": (C.c_int, [_P, _P, _P, _P, _P]),
    "sem_pressure_apply_f32": (C.c_int, [_P, _P, _P, _P, _P]),
    "sem_pressure_solve": (C.c_int, [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
}

_lib = None


def lib():
    """Load libsem.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, what):
    if status != SEM_OK:
        msg = lib().sem_last_error().decode(errors="replace")
        name = lib().sem_status_str(status).decode()
        raise SemError(status, f"{what}: {name}: {msg}")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype=None, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype, numel=None):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy {dtype} array")
    if numel is not None and a.size != numel:
        raise ValueError(f"expected {numel} elements, got {a.size}")
    return C.c_void_p(a.ctypes.data)


def make_desc(desc):
    """Fill a MeshDesc from a dict (keys as in sem_mesh_desc; 'kind' is
    'box', 'pipe' or 'explicit').  Returns (MeshDesc, keepalive list)."""
    d = MeshDesc()
    keep = []
    d.kind = KIND[desc["kind"]]
    d.N = int(desc["N"])
    if desc["kind"] == "box":
        d.nx, d.ny, d.nz = int(desc["nx"]), int(desc["ny"]), int(desc["nz"])
        d.lx, d.ly, d.lz = float(desc.get("lx", 1.0)), float(desc.get("ly", 1.0)), float(desc.get("lz", 1.0))
    elif desc["kind"] == "pipe":
        d.nc, d.nr, d.nzp = int(desc["nc"]), int(desc["nr"]), int(desc["nzp"])
        d.R, d.L = float(desc.get("R", 1.0)), float(desc.get("L", 8.0))
        d.a = float(desc.get("a", 0.5 * d.R))
        d.beta = float(desc.get("beta", 2.0))
        d.periodic_z = int(bool(desc.get("periodic", True)))
    else:
        xyz = np.ascontiguousarray(desc["xyz"], dtype=np.float64)
        vert = np.ascontiguousarray(desc["vert"], dtype=np.int64)
        dface = np.ascontiguousarray(desc["dirichlet_face"], dtype=np.uint8)
        d.E = int(vert.shape[0])
        d.xyz, d.vert, d.dirichlet_face = xyz.ctypes.data, vert.ctypes.data, dface.ctypes.data
        keep += [xyz, vert, dface]
    return d, keep


def _opts(tol=1e-10, h1=1.0, h2=0.0, prec=FP64, inner_tol=0.0, maxit=0, max_outer=0, refine=0, delta=0.0,
          precond=0):
    o = SolveOpts()
    o.tol, o.h1, o.h2, o.inner_tol = float(tol), float(h1), float(h2), float(inner_tol)
    o.maxit, o.max_outer, o.prec = int(maxit), int(max_outer), int(prec)
    o.refine, o.delta, o.precond = int(refine), float(delta), int(precond)
    return o


class Mesh:
    """A mesh resident on the current CUDA device (sem_mesh_create)."""

    def __init__(self, desc, stream=None):
        d, keep = make_desc(desc)
        h = C.c_void_p()
        _check(lib().sem_mesh_create(C.byref(d), _stream(stream), C.byref(h)), "sem_mesh_create")
        self._h = h
        info = MeshInfo()
        _check(lib().sem_mesh_info(h, C.byref(info)), "sem_mesh_info")
        self.E, self.N, self.n_local, self.n_global = info.E, info.N, info.n_local, info.n_global
        self.n_segments, self.n_seg_points, self.dev_bytes = info.n_segments, info.n_seg_points, info.dev_bytes
        self.n = self.N + 1
        self.shape = (self.E, self.n, self.n, self.n)

    def close(self):
        if getattr(self, "_h", None):
            lib().sem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fp64_double_float(self):
        """True if FP64 requests on this mesh run the double-float kernel."""
        return bool(lib().sem_mesh_fp64_kernel(self._h))

    def check(self, stream=None):
        """sem_mesh_check: raise if a bounded device-side wait gave up."""
        _check(lib().sem_mesh_check(self._h, _stream(stream)), "sem_mesh_check")

    def ax_variant(self, prec=FP32):
        """Kernel variant the autotuner chose for `prec` (0/1 register kernels, 2/3 bulk-copy pipelined)."""
        return int(lib().sem_mesh_ax_variant(self._h, int(prec)))

    def global_ids(self):
        out = np.empty(self.n_local, dtype=np.int64)
        _check(lib().sem_mesh_global_ids(self._h, out.ctypes.data), "sem_mesh_global_ids")
        return out

    def coords(self, stream=None):
        import torch
        out = torch.empty((self.E, 3, self.n, self.n, self.n), dtype=torch.float64, device="cuda")
        _check(lib().sem_mesh_coords(self._h, _dptr(out), _stream(stream)), "sem_mesh_coords")
        return out

    def geometry(self, stream=None):
        import torch
        G = torch.empty((self.E, 6, self.n, self.n, self.n), dtype=torch.float64, device="cuda")
        B = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(lib().sem_mesh_geometry(self._h, _dptr(G), _dptr(B), _stream(stream)), "sem_mesh_geometry")
        return G, B

    def set_coefficients(self, h1=None, h2=None, stream=None):
        """sem_mesh_set_coefficients: per-point h1, h2 (device FP64 tensors of
        n_local values, local layout) multiplying the scalar h1, h2 of every
        later operator call; None means 1 everywhere (both None: constant
        coefficients again)."""
        import torch
        p1 = _dptr(h1, torch.float64, self.n_local) if h1 is not None else None
        p2 = _dptr(h2, torch.float64, self.n_local) if h2 is not None else None
        _check(lib().sem_mesh_set_coefficients(self._h, p1, p2, _stream(stream)), "sem_mesh_set_coefficients")

    def weights(self, stream=None):
        import torch
        mult = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        mask = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        _check(lib().sem_mesh_weights(self._h, _dptr(mult), _dptr(mask), _stream(stream)), "sem_mesh_weights")
        return mult, mask

    def ax(self, u, w, h1=1.0, h2=0.0, prec=FP64, stream=None):
        import torch
        dt = torch.float64 if prec == FP64 else torch.float32
        _check(lib().sem_ax(self._h, _dptr(u, dt, self.n_local), _dptr(w, dt, self.n_local), float(h1), float(h2),
                            int(prec), _stream(stream)), "sem_ax")
        return w

    def gs(self, v, apply_mask=True, prec=FP64, stream=None):
        import torch
        dt = torch.float64 if prec == FP64 else torch.float32
        _check(lib().sem_gs(self._h, _dptr(v, dt, self.n_local), int(prec), int(bool(apply_mask)), _stream(stream)),
               "sem_gs")
        return v

    def rhs(self, f, b, stream=None):
        import torch
        _check(lib().sem_rhs(self._h, _dptr(f, torch.float64, self.n_local), _dptr(b, torch.float64, self.n_local),
                             _stream(stream)), "sem_rhs")
        return b

    def apply(self, x, y, h1=1.0, h2=0.0, stream=None):
        import torch
        _check(lib().sem_apply(self._h, _dptr(x, torch.float64, self.n_local), _dptr(y, torch.float64, self.n_local),
                               float(h1), float(h2), _stream(stream)), "sem_apply")
        return y

    def jacobi(self, out, h1=1.0, h2=0.0, stream=None):
        import torch
        _check(lib().sem_jacobi(self._h, float(h1), float(h2), _dptr(out, torch.float64, self.n_local),
                                _stream(stream)), "sem_jacobi")
        return out

    # -- staggered P_N - P_{N-2} pressure space (Sec. 2, Eq. 5) -------------
    @property
    def pressure_shape(self):
        """Shape of a pressure field: (E, m, m, m), m = N - 1."""
        return (self.E,) + (self.N - 1,) * 3

    def pressure_size(self):
        v = C.c_int64()
        _check(lib().sem_pressure_info(self._h, C.byref(v)), "sem_pressure_info")
        return v.value

    def pressure_factors(self, stream=None):
        """GL-point factors F [E, 9, m, m, m] (entry 3 b + a = rho^3 adj(J)_{ba})."""
        import torch
        m = self.N - 1
        F = torch.empty((self.E, 9, m, m, m), dtype=torch.float64, device="cuda")
        _check(lib().sem_pressure_factors(self._h, _dptr(F), _stream(stream)), "sem_pressure_factors")
        return F

    def pressure_grad(self, p, u, stream=None):
        """u = D^T p: p [E, m, m, m] -> u [3, E, n, n, n] (local, unassembled)."""
        import torch
        _check(lib().sem_pressure_grad(self._h, _dptr(p, torch.float64, self.pressure_size()),
                                       _dptr(u, torch.float64, 3 * self.n_local), _stream(stream)),
               "sem_pressure_grad")
        return u

    def pressure_div(self, u, q, stream=None):
        """q = D u: u [3, E, n, n, n] -> q [E, m, m, m] (element by element)."""
        import torch
        _check(lib().sem_pressure_div(self._h, _dptr(u, torch.float64, 3 * self.n_local),
                                      _dptr(q, torch.float64, self.pressure_size()), _stream(stream)),
               "sem_pressure_div")
        return q

    def pressure_apply(self, p, q, work=None, stream=None):
        """q = E p = D B^{-1} D^T p; work: 3 n_local doubles of scratch (allocated if None)."""
        import torch
        if work is None:
            work = torch.empty(3 * self.n_local, dtype=torch.float64, device="cuda")
        np_ = self.pressure_size()
        _check(lib().sem_pressure_apply(self._h, _dptr(p, torch.float64, np_), _dptr(q, torch.float64, np_),
                                        _dptr(work, torch.float64, 3 * self.n_local), _stream(stream)),
               "sem_pressure_apply")
        return q

    def pressure_apply_f32(self, p, q, work=None, stream=None):
        """q = E p in FP32 (sem_pressure_apply_f32); work: 3 n_local floats (allocated if None)."""
        import torch
        if work is None:
            work = torch.empty(3 * self.n_local, dtype=torch.float32, device="cuda")
        np_ = self.pressure_size()
        _check(lib().sem_pressure_apply_f32(self._h, _dptr(p, torch.float32, np_), _dptr(q, torch.float32, np_),
                                            _dptr(work, torch.float32, 3 * self.n_local), _stream(stream)),
               "sem_pressure_apply_f32")
        return q

    def pressure_diag(self, d, stream=None):
        """sem_pressure_diag: diag(E) into the FP64 device tensor d [E, m, m, m]."""
        import torch
        _check(lib().sem_pressure_diag(self._h, _dptr(d, torch.float64, self.pressure_size()), _stream(stream)),
               "sem_pressure_diag")

    def pressure_solve(self, g, p, tol=1e-10, maxit=0, stream=None, check=False, prec=FP64, delta=0.0,
                       precond=PRECOND_DEFAULT):
        """sem_pressure_solve: E p = g on the mean-free pressure space (CG,
        Jacobi-preconditioned unless precond=PRECOND_NONE; prec=MIXED: FP32
        operator with FP64 reliable updates); returns the result record (a
        dict), raising on errors other than not-converged / breakdown unless
        check=True."""
        import torch
        o = _opts(tol=tol, maxit=maxit, prec=prec, delta=delta, precond=precond)
        r = SolveResult()
        np_ = self.pressure_size()
        st = lib().sem_pressure_solve(self._h, _dptr(g, torch.float64, np_), _dptr(p, torch.float64, np_),
                                      C.byref(o), C.byref(r), _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN) or (check and st != SEM_OK):
            _check(st, "sem_pressure_solve")
        return r.as_dict()

    def solve(self, b, x, stream=None, check=False, **opts):
        """sem_pcg_solve on device tensors; returns the result record (a dict).
        A non-converged / breakdown status is reported in the record; with
        check=True it raises instead."""
        import torch
        o = _opts(**opts)
        r = SolveResult()
        st = lib().sem_pcg_solve(self._h, _dptr(b, torch.float64, self.n_local), _dptr(x, torch.float64, self.n_local),
                                 C.byref(o), C.byref(r), _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN) or (check and st != SEM_OK):
            _check(st, "sem_pcg_solve")
        return r.as_dict()

    def solve_noalloc(self, b, x, stream=None, **opts):
        """sem_pcg_solve_noalloc: the FP64 solve with all scratch in the
        library's fixed device array (no device allocation in the call)."""
        import torch
        o = _opts(**opts)
        r = SolveResult()
        st = lib().sem_pcg_solve_noalloc(self._h, _dptr(b, torch.float64, self.n_local),
                                         _dptr(x, torch.float64, self.n_local), C.byref(o), C.byref(r),
                                         _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN):
            _check(st, "sem_pcg_solve_noalloc")
        return r.as_dict()

    def solve_host(self, b, x, stream=None, **opts):
        """sem_pcg_solve_host on numpy float64 arrays (copies inside the call)."""
        o = _opts(**opts)
        r = SolveResult()
        st = lib().sem_pcg_solve_host(self._h, _hptr(b, np.float64, self.n_local), _hptr(x, np.float64, self.n_local),
                                      C.byref(o), C.byref(r), _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN):
            _check(st, "sem_pcg_solve_host")
        return r.as_dict()


def solve_batch(meshes, bs, xs, opts_list=None, stream=None, **opts):
    """sem_pcg_solve_batch: mixed-precision solves of one odd order N together.
    meshes, bs, xs: lists (CUDA float64 tensors); opts_list: per-request dicts
    (defaults to the keyword options for all).  Returns (status, [result dicts])."""
    import torch
    k = len(meshes)
    if opts_list is None:
        opts_list = [opts] * k
    Mh = (C.c_void_p * k)(*[m._h.value for m in meshes])
    Bp = (C.c_void_p * k)(*[_dptr(b, torch.float64, m.n_local).value for b, m in zip(bs, meshes)])
    Xp = (C.c_void_p * k)(*[_dptr(x, torch.float64, m.n_local).value for x, m in zip(xs, meshes)])
    Op = (SolveOpts * k)(*[_opts(**dict({"prec": MIXED}, **o)) for o in opts_list])
    Rs = (SolveResult * k)()
    st = lib().sem_pcg_solve_batch(Mh, Bp, Xp, Op, Rs, k, _stream(stream))
    if st in (SEM_ERR_INVALID, SEM_ERR_CUDA, SEM_ERR_OOM):
        _check(st, "sem_pcg_solve_batch")
    return st, [Rs[q].as_dict() for q in range(k)]


def kernel_launches():
    """Kernels launched by the library so far in this process (graph replays
    count every kernel node)."""
    return int(lib().sem_kernel_launches())


def topology_numbering(E, N, vert):
    """Host-only: first-touch global ids from corner vertex ids (sem_topology_numbering)."""
    vert = np.ascontiguousarray(vert, dtype=np.int64)
    out = np.empty(E * (N + 1) ** 3, dtype=np.int64)
    ng = C.c_int64()
    _check(lib().sem_topology_numbering(int(E), int(N), vert.ctypes.data, out.ctypes.data, C.byref(ng)),
           "sem_topology_numbering")
    return out, ng.value


def gs_halo(E, N, vert, elem_rank, rank):
    """Host-only (sem_gs_halo): the halo of `rank` under the element partition
    elem_rank [E].  Returns (node_gid, node_ptr, copy_rank, copy_local)."""
    vert = np.ascontiguousarray(vert, dtype=np.int64)
    er = np.ascontiguousarray(elem_rank, dtype=np.int32)
    nn, nc = C.c_int64(), C.c_int64()
    _check(lib().sem_gs_halo(int(E), int(N), vert.ctypes.data, er.ctypes.data, int(rank), C.byref(nn), C.byref(nc),
                             None, None, None, None), "sem_gs_halo")
    gid = np.empty(nn.value, dtype=np.int64)
    ptr = np.empty(nn.value + 1, dtype=np.int64)
    crank = np.empty(nc.value, dtype=np.int32)
    cloc = np.empty(nc.value, dtype=np.int64)
    _check(lib().sem_gs_halo(int(E), int(N), vert.ctypes.data, er.ctypes.data, int(rank), C.byref(nn), C.byref(nc),
                             gid.ctypes.data, ptr.ctypes.data, crank.ctypes.data, cloc.ctypes.data), "sem_gs_halo")
    return gid, ptr, crank, cloc


def mesh_vertices(desc):
    """Host-only: corner vertex ids [E, 8] of the built-in generators."""
    d, keep = make_desc(desc)
    E = C.c_int64()
    _check(lib().sem_mesh_vertices(C.byref(d), None, C.byref(E)), "sem_mesh_vertices")
    out = np.empty((E.value, 8), dtype=np.int64)
    _check(lib().sem_mesh_vertices(C.byref(d), out.ctypes.data, C.byref(E)), "sem_mesh_vertices")
    return out


class Projection:
    """Projection space of earlier solutions for one mesh and one operator
    (sem_proj_*): solve() starts CG from the projection of b onto the space
    and adds the new direction to it."""

    def __init__(self, mesh, max_vectors=8, h1=1.0, h2=0.0):
        h = C.c_void_p()
        _check(lib().sem_proj_create(mesh._h, int(max_vectors), float(h1), float(h2), C.byref(h)), "sem_proj_create")
        self._h, self.mesh, self.h1, self.h2 = h, mesh, float(h1), float(h2)

    def solve(self, b, x, stream=None, check=False, **opts):
        import torch
        opts.setdefault("h1", self.h1)
        opts.setdefault("h2", self.h2)
        o = _opts(**opts)
        r = SolveResult()
        n = self.mesh.n_local
        st = lib().sem_proj_solve(self._h, _dptr(b, torch.float64, n), _dptr(x, torch.float64, n), C.byref(o),
                                  C.byref(r), _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN) or (check and st != SEM_OK):
            _check(st, "sem_proj_solve")
        return r.as_dict()

    def size(self):
        k = C.c_int()
        _check(lib().sem_proj_size(self._h, C.byref(k)), "sem_proj_size")
        return k.value

    def reset(self):
        _check(lib().sem_proj_reset(self._h), "sem_proj_reset")

    def close(self):
        if getattr(self, "_h", None):
            lib().sem_proj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SCHWARZ_COARSE = 1
SCHWARZ_FP32_PRECOND = 2
SCHWARZ_DENSE_COARSE_MAX = 8192


class Schwarz:
    """Overlapping Schwarz preconditioner of one mesh and operator
    (sem_schwarz_*): fast-diagonalisation local solves on the elements with
    the symmetric mult^-1/2 weights, plus the trilinear coarse grid."""

    def __init__(self, mesh, h1=1.0, h2=0.0, coarse=True, fp32_precond=False):
        h = C.c_void_p()
        flags = (SCHWARZ_COARSE if coarse else 0) | (SCHWARZ_FP32_PRECOND if fp32_precond else 0)
        _check(lib().sem_schwarz_create(mesh._h, float(h1), float(h2), flags, C.byref(h)), "sem_schwarz_create")
        self._h, self.mesh, self.h1, self.h2 = h, mesh, float(h1), float(h2)

    def info(self):
        i = SchwarzInfo()
        _check(lib().sem_schwarz_info(self._h, C.byref(i)), "sem_schwarz_info")
        return {"n_distinct": i.n_distinct, "n_coarse": i.n_coarse, "coarse": int(i.coarse),
                "dev_bytes": i.dev_bytes, "setup_ms": i.setup_ms}

    def apply(self, r, z, prec=FP64, stream=None):
        import torch
        dt = torch.float32 if prec == FP32 else torch.float64
        n = self.mesh.n_local
        _check(lib().sem_schwarz_apply(self._h, _dptr(r, dt, n), _dptr(z, dt, n), int(prec), _stream(stream)),
               "sem_schwarz_apply")

    def solve(self, b, x, stream=None, check=False, **opts):
        import torch
        opts.setdefault("h1", self.h1)
        opts.setdefault("h2", self.h2)
        o = _opts(**opts)
        r = SolveResult()
        n = self.mesh.n_local
        st = lib().sem_schwarz_solve(self._h, _dptr(b, torch.float64, n), _dptr(x, torch.float64, n), C.byref(o),
                                     C.byref(r), _stream(stream))
        if st not in (SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN) or (check and st != SEM_OK):
            _check(st, "sem_schwarz_solve")
        return r.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().sem_schwarz_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server (sem_server_*)."""

    def __init__(self, hbm_budget_bytes=0, max_slots=8, max_queue=4096, device=0, batch=True):
        o = ServerOpts()
        o.hbm_budget_bytes, o.max_slots, o.max_queue, o.device = int(hbm_budget_bytes), max_slots, max_queue, device
        o.batch = 0 if batch else 1
        h = C.c_void_p()
        _check(lib().sem_server_create(C.byref(o), C.byref(h)), "sem_server_create")
        self._h = h

    def submit(self, desc, f, **opts):
        d, keep = make_desc(desc)
        f = np.ascontiguousarray(f, dtype=np.float64)
        o = _opts(**opts)
        rid = C.c_uint64()
        _check(lib().sem_server_submit(self._h, C.byref(d), f.ctypes.data, C.byref(o), C.byref(rid)),
               "sem_server_submit")
        return rid.value

    def poll(self, rid, timeout_ms=-1, n_local=None, timing=False):
        """Returns (status, x or None, result dict); status SEM_ERR_TIMEOUT if
        not done.  With timing=True the result dict also carries the request's
        latency breakdown (sem_server_poll_timed) under "timing"."""
        r = SolveResult()
        tm = RequestTiming()
        x = np.empty(n_local, dtype=np.float64) if n_local else None
        st = lib().sem_server_poll_timed(self._h, C.c_uint64(rid), int(timeout_ms),
                                         x.ctypes.data if x is not None else None, C.byref(r),
                                         C.byref(tm) if timing else None)
        if st in (SEM_ERR_INVALID, SEM_ERR_NOT_FOUND, SEM_ERR_CUDA, SEM_ERR_OOM):
            _check(st, "sem_server_poll")
        out = r.as_dict()
        if timing and st != SEM_ERR_TIMEOUT:
            out["timing"] = {k: getattr(tm, k) for k, _ in RequestTiming._fields_}
        return st, (x if st not in (SEM_ERR_TIMEOUT,) else None), out

    def cancel(self, rid):
        return lib().sem_server_cancel(self._h, C.c_uint64(rid))

    def stats(self):
        s = ServerStats()
        _check(lib().sem_server_stats_get(self._h, C.byref(s)), "sem_server_stats_get")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().sem_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pressure_basis(N):
    """sem_pressure_basis (host only): (zeta [m], rho [m], Ig [m, n], DIg [m, n])
    of the P_N - P_{N-2} pressure space, m = N - 1, n = N + 1."""
    m, n = N - 1, N + 1
    if m < 1:
        _check(lib().sem_pressure_basis(int(N), None, None, None, None), "sem_pressure_basis")
    z, r = np.empty(m), np.empty(m)
    Ig, DIg = np.empty((m, n)), np.empty((m, n))
    _check(lib().sem_pressure_basis(int(N), z.ctypes.data, r.ctypes.data, Ig.ctypes.data, DIg.ctypes.data),
           "sem_pressure_basis")
    return z, r, Ig, DIg


def schwarz_fdm_1d(N, l, l_lo=None, l_hi=None, dir_lo=False, dir_hi=False):
    """sem_schwarz_fdm_1d (host only): (S [n, n], lam [n]) of one 1D problem."""
    n = N + 1
    S, lam = np.empty((n, n)), np.empty(n)
    _check(lib().sem_schwarz_fdm_1d(int(N), float(l), float(l_lo or 0.0), float(l_hi or 0.0), int(bool(dir_lo)),
                                    int(bool(dir_hi)), S.ctypes.data, lam.ctypes.data), "sem_schwarz_fdm_1d")
    return S, lam


def schwarz_setup_host(N, glo, xyz, dirichlet_face):
    """sem_schwarz_setup_host: (S [E, 3, n, n], lam [E, 3, n], distinct count)
    from host arrays glo [E*n^3] int64, xyz [E, 3, n, n, n], dirichlet_face [E, 6]."""
    glo = np.ascontiguousarray(glo, dtype=np.int64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    df = np.ascontiguousarray(dirichlet_face, dtype=np.uint8)
    E, n = xyz.shape[0], N + 1
    S, lam = np.empty((E, 3, n, n)), np.empty((E, 3, n))
    k = C.c_int64()
    _check(lib().sem_schwarz_setup_host(int(E), int(N), glo.ctypes.data, xyz.ctypes.data, df.ctypes.data,
                                        S.ctypes.data, lam.ctypes.data, C.byref(k)), "sem_schwarz_setup_host")
    return S, lam, k.value

