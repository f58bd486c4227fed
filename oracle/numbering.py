"""Global numbering, direct stiffness summation QQ^T and the Dirichlet mask.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2 separates the global operation (the "exchange of element face
values": summing the contributions of all element-local copies of a shared
GLL node) from the local tensor-product work.  The paper does not define the
numbering; the reading taken here:

* Two local points are the same global node when they coincide in space
  (after identifying z = 0 with z = L for a periodic pipe).  The oracle finds
  coincident points geometrically, with a k-d tree and a tolerance far below
  the smallest GLL spacing -- a different route from the library's
  topological (vertex/edge/face) construction; both must give the same
  partition.
* Global ids are assigned in order of first appearance when the local points
  are scanned in ascending local index l = i + n (j + n (k + n e)).
* QQ^T: every node's value is the sum of its copies taken in ascending local
  index, left to right; the sum is written back to every copy.
"""

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

# Points closer than this are the same node.  GLL spacing on the meshes used
# here is >= 1e-4, coordinate round-off ~1e-15.
COINCIDENCE_TOL = 1e-9


def local_points(mesh):
    """[P_L, 3] coordinates in local-index order (i fastest, then j, k, e)."""
    return mesh.xyz.transpose(0, 2, 3, 4, 1).reshape(-1, 3)


def global_numbering(mesh, tol=COINCIDENCE_TOL):
    """Return (glo[P_L] int64, P_G): first-touch global ids of all local points."""
    pts = local_points(mesh).copy()
    if mesh.period is not None:
        top = pts[:, 2] >= mesh.period - tol
        pts[top, 2] -= mesh.period
    P = pts.shape[0]
    pairs = cKDTree(pts).query_pairs(tol, output_type="ndarray")
    graph = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(P, P))
    ncomp, comp = connected_components(graph, directed=False)
    first = np.full(ncomp, P, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(P, dtype=np.int64))
    rank = np.empty(ncomp, dtype=np.int64)
    rank[np.argsort(first, kind="stable")] = np.arange(ncomp, dtype=np.int64)
    return rank[comp], int(ncomp)


def multiplicity(glo, Pg):
    """Number of local copies of each local point's node."""
    return np.bincount(glo, minlength=Pg)[glo]


def face_points(n, face):
    """Boolean [n, n, n] (k, j, i) selector of the points on one element face."""
    sel = np.zeros((n, n, n), dtype=bool)
    if face == 0:
        sel[:, :, 0] = True
    elif face == 1:
        sel[:, :, n - 1] = True
    elif face == 2:
        sel[:, 0, :] = True
    elif face == 3:
        sel[:, n - 1, :] = True
    elif face == 4:
        sel[0, :, :] = True
    else:
        sel[n - 1, :, :] = True
    return sel


def dirichlet_mask(mesh, glo, Pg):
    """1.0 on free nodes, 0.0 on every copy of a node that lies on a Dirichlet
    face of any element."""
    n = mesh.n
    on_face = np.zeros((mesh.E, n, n, n), dtype=bool)
    for f in range(6):
        sel = face_points(n, f)
        on_face[mesh.dirichlet_face[:, f]] |= sel
    dnode = np.zeros(Pg, dtype=bool)
    dnode[glo[on_face.reshape(-1)]] = True
    return np.where(dnode[glo], 0.0, 1.0)


def gs(v, glo, Pg):
    """QQ^T v for a local field of any shape (flattened in local order).

    np.add.at applies its additions one index at a time in the order of the
    index array, so each node's sum runs over its copies in ascending local
    index, starting from 0.0 (0.0 + x == x, up to the sign of a zero)."""
    flat = np.asarray(v).reshape(-1)
    s = np.zeros(Pg, dtype=flat.dtype)
    np.add.at(s, glo, flat)
    return s[glo].reshape(np.shape(v))


def gs_loop(v, glo, Pg):
    """The same sum as ``gs`` written as a plain loop (small inputs only)."""
    flat = np.asarray(v).reshape(-1)
    s = [None] * Pg
    for l, g in enumerate(glo):
        s[g] = flat[l] if s[g] is None else s[g] + flat[l]
    return np.array([s[g] for g in glo], dtype=flat.dtype).reshape(np.shape(v))
