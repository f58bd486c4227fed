"""Synthetic hexahedral meshes: a box and an O-grid straight pipe.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2: the domain is split into non-overlapping, body-conforming hexahedra;
Sec. 4.2: the paper's flow case is a straight periodic pipe (237,120 and
853,632 elements).  Those meshes are not available, so a synthetic O-grid
pipe stands in for them:

* a central square of half-width ``a`` with nc x nc elements;
* four curved blocks of nc (tangential) x nr (radial) elements around it.  In
  the block on the +x side a point with tangential coordinate s in [-1, 1] and
  radial coordinate t in [0, 1] sits at
  (1 - t) (a, a s) + t R (cos(pi s / 4), sin(pi s / 4));
  the other three blocks are that block rotated by 90, 180 and 270 degrees;
* radial levels clustered toward the wall: t_k = 1 - tanh(beta (1 - k/nr)) / tanh(beta);
* nzp uniform layers in z on [0, L], periodic in z by default.

GLL point coordinates are the analytic map evaluated at each element's GLL
reference coordinates, so the outer elements are curved and non-affine.

Array conventions (shared by the whole oracle): an element-local field is an
array of shape [E, n, n, n] indexed [e, k, j, i] (i fastest in memory, the
layout of Alg. 1's u(i,j,k,e)); coordinates are [E, 3, n, n, n].
Element faces are numbered 0: i=0, 1: i=N, 2: j=0, 3: j=N, 4: k=0, 5: k=N.
"""

import numpy as np

from . import gll


class Mesh:
    """Nodal coordinates plus the boundary description of one mesh."""

    def __init__(self, N, xyz, dirichlet_face, period=None, kind="explicit"):
        self.N = int(N)
        self.n = self.N + 1
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.E = self.xyz.shape[0]
        self.dirichlet_face = np.asarray(dirichlet_face, dtype=bool)
        self.period = period  # None, or the z-period length (periodic in z)
        self.kind = kind


def _lerp(a, b, xi):
    """Point at reference coordinate xi in [-1, 1] of the segment [a, b];
    exact at both ends."""
    return a * (1.0 - xi) * 0.5 + b * (1.0 + xi) * 0.5


def box(nx, ny, nz, N, lx=1.0, ly=1.0, lz=1.0, elements=None):
    """Affine box [0,lx]x[0,ly]x[0,lz] with nx*ny*nz elements, element index
    e = ex + nx (ey + ny ez), Dirichlet on all six faces.  ``elements``
    (optional index array) builds only those elements, in that order."""
    xi, _ = gll.nodes_weights(N)
    n = N + 1
    e = np.arange(nx * ny * nz) if elements is None else np.asarray(elements)
    E = e.size
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    x = _lerp((lx * ex / nx)[:, None], (lx * (ex + 1) / nx)[:, None], xi[None, :])  # [E, n] over i
    y = _lerp((ly * ey / ny)[:, None], (ly * (ey + 1) / ny)[:, None], xi[None, :])  # over j
    z = _lerp((lz * ez / nz)[:, None], (lz * (ez + 1) / nz)[:, None], xi[None, :])  # over k
    xyz = np.empty((E, 3, n, n, n))
    xyz[:, 0] = x[:, None, None, :]
    xyz[:, 1] = y[:, None, :, None]
    xyz[:, 2] = z[:, :, None, None]
    dface = np.zeros((E, 6), dtype=bool)
    dface[:, 0] = ex == 0
    dface[:, 1] = ex == nx - 1
    dface[:, 2] = ey == 0
    dface[:, 3] = ey == ny - 1
    dface[:, 4] = ez == 0
    dface[:, 5] = ez == nz - 1
    return Mesh(N, xyz, dface, None, "box")


def pipe_radial_levels(nr, beta):
    """t_k = 1 - tanh(beta (1 - k/nr)) / tanh(beta), k = 0..nr (t_0 = 0, t_nr = 1)."""
    k = np.arange(nr + 1)
    return 1.0 - np.tanh(beta * (1.0 - k / nr)) / np.tanh(beta)


def _rotate(px, py, q):
    """Rotate (px, py) by q quarter turns counter-clockwise."""
    if q == 0:
        return px, py
    if q == 1:
        return -py, px
    if q == 2:
        return -px, -py
    return py, -px


def pipe(nc, nr, nzp, N, R=1.0, L=8.0, a=None, beta=2.0, periodic=True, elements=None):
    """O-grid straight pipe of radius R and length L (see module docstring).

    Element order: e = layer * n2d + e2d, n2d = nc (nc + 4 nr).  In a layer the
    central-square elements come first (e2d = ey nc + ex; local i along x, j
    along y), then blocks q = 0..3 (e2d = nc^2 + q nc nr + r nc + m, m the
    tangential and r the radial index; local i runs outward (t), j along the
    tangential coordinate s, which keeps every element right-handed).  Local k
    runs along z.  Dirichlet: the wall face (i = N of the outermost ring), and
    the end caps when the pipe is not periodic.  ``elements`` (optional index
    array) builds only those elements, in that order.
    """
    if a is None:
        a = 0.5 * R
    xi, _ = gll.nodes_weights(N)
    n = N + 1
    n2d = nc * (nc + 4 * nr)
    E = n2d * nzp
    tlev = pipe_radial_levels(nr, beta)
    xy = np.empty((n2d, 2, n, n))  # [e2d, comp, j, i]
    wall = np.zeros(n2d, dtype=bool)
    XI_i = xi[None, :]  # varies along i (last axis)
    XI_j = xi[:, None]  # varies along j
    for ey in range(nc):
        for ex in range(nc):
            e2 = ey * nc + ex
            xa, xb = -a + 2.0 * a * ex / nc, -a + 2.0 * a * (ex + 1) / nc
            ya, yb = -a + 2.0 * a * ey / nc, -a + 2.0 * a * (ey + 1) / nc
            xy[e2, 0] = _lerp(xa, xb, XI_i) + 0.0 * XI_j
            xy[e2, 1] = _lerp(ya, yb, XI_j) + 0.0 * XI_i
    for q in range(4):
        for r in range(nr):
            for m in range(nc):
                e2 = nc * nc + q * nc * nr + r * nc + m
                t = _lerp(tlev[r], tlev[r + 1], XI_i) + 0.0 * XI_j
                s = _lerp(-1.0 + 2.0 * m / nc, -1.0 + 2.0 * (m + 1) / nc, XI_j) + 0.0 * XI_i
                th = s * np.pi / 4.0
                px = (1.0 - t) * a + t * R * np.cos(th)
                py = (1.0 - t) * a * s + t * R * np.sin(th)
                xy[e2, 0], xy[e2, 1] = _rotate(px, py, q)
                wall[e2] = r == nr - 1
    eidx = np.arange(E) if elements is None else np.asarray(elements)
    E = eidx.size
    layer = eidx // n2d
    e2d = eidx % n2d
    z = _lerp((L * layer / nzp)[:, None], (L * (layer + 1) / nzp)[:, None], xi[None, :])  # [E, k]
    xyz = np.empty((E, 3, n, n, n))
    xyz[:, 0] = xy[e2d, 0][:, None, :, :]
    xyz[:, 1] = xy[e2d, 1][:, None, :, :]
    xyz[:, 2] = z[:, :, None, None]
    dface = np.zeros((E, 6), dtype=bool)
    dface[:, 1] = wall[e2d]
    if not periodic:
        dface[:, 4] = layer == 0
        dface[:, 5] = layer == nzp - 1
    return Mesh(N, xyz, dface, L if periodic else None, "pipe")


def pipe_global_node_count(nc, nr, nzp, N, periodic=True):
    """Closed form for the number of distinct GLL nodes of the pipe: the
    cross-section holds (nc N + 1)^2 square nodes plus 4 nc N nodes on each of
    the nr N radial levels outside the square; z holds nzp N levels if
    periodic, nzp N + 1 otherwise."""
    p2 = (nc * N + 1) ** 2 + 4 * nc * nr * N * N
    return p2 * (nzp * N if periodic else nzp * N + 1)


def box_global_node_count(nx, ny, nz, N):
    return (nx * N + 1) * (ny * N + 1) * (nz * N + 1)
