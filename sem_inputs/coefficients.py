"""Seeded per-point operator coefficients h1(i,j,k,e) and h2(i,j,k,e).

A variable-viscosity Helmholtz step: h1 = nu(x) > 0, smooth in space, times a
seeded per-element factor (a coefficient read per local point need not be
continuous across element faces); h2 = (b0/dt) rho(x) > 0, smooth.  Both are
returned on the local layout [E, n, n, n] (k, j, i per element) from the
nodal coordinates xyz [E, 3, n, n, n].
"""

import numpy as np


def _smooth(rng, xyz, amp):
    k = rng.uniform(0.5, 2.0, 3)
    ph = rng.uniform(0.0, 2.0 * np.pi, 3)
    s = np.ones(xyz.shape[:1] + xyz.shape[2:])
    for a in range(3):
        s = s * np.sin(k[a] * xyz[:, a] + ph[a])
    return 1.0 + amp * s


def viscosity(seed, xyz, nu0=1.0, amp=0.5, jump=0.2):
    """h1 in [nu0 (1-amp)(1-jump), nu0 (1+amp)(1+jump)]."""
    rng = np.random.default_rng(seed)
    smooth = _smooth(rng, xyz, amp)
    per_element = 1.0 + jump * rng.uniform(-1.0, 1.0, xyz.shape[0])
    return nu0 * smooth * per_element[:, None, None, None]


def mass_coefficient(seed, xyz, c0=10.0, amp=0.3):
    """h2 in [c0 (1-amp), c0 (1+amp)]."""
    rng = np.random.default_rng(seed)
    return c0 * _smooth(rng, xyz, amp)
