"""Seeded request stream for the serving workload.

Each request is a Poisson or Helmholtz solve on a box or pipe mesh:
log2 E_target ~ U[9, 15] snapped to the nearest achievable near-cubic box or pipe, box/pipe
50/50, N uniform in {5, 7, 9}, Poisson/Helmholtz 50/50 with h1 = 1 and
h2 log-uniform in [1e-2, 1e2], Poisson-process arrivals at ``rate`` per
second, forcing from ``forcing.random_modes`` with a per-request seed.
"""

import math

import numpy as np

# Pipe cross-sections (nc, nr) and their element counts per layer.
_PIPE_XS = [(2, 1), (4, 1), (4, 2), (8, 2)]


def _box_near(E):
    """Near-cubic nx <= ny <= nz <= 2 nx on the unit cube (elements of aspect
    ratio <= 2) with nx*ny*nz closest to E."""
    best = None
    for nx in range(1, 64):
        for ny in range(nx, 2 * nx + 1):
            nz = max(ny, min(2 * nx, round(E / (nx * ny))))
            cand = nx * ny * nz
            err = abs(math.log(cand / E))
            if best is None or err < best[0]:
                best = (err, dict(kind="box", nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.0, lz=1.0))
    return best[1]


def _pipe_near(E):
    best = None
    for nc, nr in _PIPE_XS:
        per = nc * (nc + 4 * nr)
        nzp = max(3, round(E / per))
        err = abs(math.log(per * nzp / E))
        if best is None or err < best[0]:
            best = (err, dict(kind="pipe", nc=nc, nr=nr, nzp=nzp, R=1.0, L=8.0, a=0.5, beta=2.0, periodic=True))
    return best[1]


def request_stream(seed, count, rate, log2_e=(9.0, 15.0), orders=(5, 7, 9)):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        E = 2.0 ** rng.uniform(*log2_e)
        desc = _box_near(E) if rng.random() < 0.5 else _pipe_near(E)
        desc["N"] = int(rng.choice(orders))
        helm = rng.random() < 0.5
        h2 = float(10.0 ** rng.uniform(-2.0, 2.0)) if helm else 0.0
        out.append(dict(id=i, arrival=t, desc=desc, h1=1.0, h2=h2, seed=int(rng.integers(1 << 31))))
    return out
