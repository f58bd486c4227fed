"""Forcing fields f evaluated at caller-supplied nodal coordinates.

* ``manufactured``: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), whose
  homogeneous-Dirichlet Poisson solution on the unit cube is
  u* = sin(pi x) sin(pi y) sin(pi z) (``manufactured_solution``).
* ``random_modes`` / ``evaluate``: a smooth seeded Gaussian-random field
  f(x) = sum_m a_m cos(k_m . x + phi_m), a_m ~ N(0, 1) / 8, integer wave
  vectors in [-4, 4]^3 scaled by (pi, pi, 2 pi / L), phi_m ~ U[0, 2 pi).
"""

import math

import numpy as np


def manufactured(xyz):
    """xyz[..., 3, ...] with the component on axis 1 (shape [E, 3, n, n, n])."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def manufactured_solution(xyz):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def random_modes(seed, L=8.0, n_modes=64):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_modes) / 8.0
    kint = rng.integers(-4, 5, size=(n_modes, 3))
    k = kint * np.array([math.pi, math.pi, 2.0 * math.pi / L])
    phi = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    return a, k, phi


def evaluate(xyz, modes):
    """numpy evaluation of the random field at coordinates [E, 3, n, n, n]."""
    a, k, phi = modes
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    f = np.zeros_like(x)
    for m in range(len(a)):
        f += a[m] * np.cos(k[m, 0] * x + k[m, 1] * y + k[m, 2] * z + phi[m])
    return f


def evaluate_torch(xyz, modes):
    """The same field with torch ops on whatever device ``xyz`` lives on (used
    to synthesise large inputs on the GPU before a timed region)."""
    import torch

    a, k, phi = modes
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    f = torch.zeros_like(x)
    for m in range(len(a)):
        f.add_(float(a[m]) * torch.cos(float(k[m, 0]) * x + float(k[m, 1]) * y
                                       + float(k[m, 2]) * z + float(phi[m])))
    return f
