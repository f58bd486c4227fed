"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of the method (no GLL points, geometry,
operator, numbering or solver): only mesh *descriptors* (sizes and shape
parameters of the box and pipe meshes), seeded random draws, the analytic
forcing fields evaluated at caller-supplied coordinates, and the request
stream of the serving workload.
"""

from .configs import MESHES, mesh_desc, elements_of  # noqa: F401
from . import forcing, vectors, serving  # noqa: F401
