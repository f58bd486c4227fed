"""Seeded random element-local fields (no continuity imposed)."""

import numpy as np


def local_field(seed, E, n, dtype=np.float64):
    """Standard-normal values on [E, n, n, n] (k, j, i order per element)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((E, n, n, n)).astype(dtype)
