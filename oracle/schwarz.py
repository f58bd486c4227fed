"""Additive overlapping Schwarz preconditioner with a coarse grid (Sec. 2, Eq. 6).

Test infrastructure only (see ``oracle/__init__``).

Eq. 6 combines local solves on overlapping subdomains, R_k^T A_k^{-1} R_k,
with a coarse-grid solve R_0^T A_0^{-1} R_0.  The paper names the method and
its coarse solver (XXT, a sparse Cholesky) but does not define the pieces.
The reading taken here, for the assembled operator A = mask QQ^T A_L of
``solver.Problem``:

* Subdomain k = element e with all its GLL nodes, including the face, edge and
  vertex nodes it shares with its neighbours (the overlap is the shared
  nodes); A_e = R_e A R_e^T is the principal submatrix of A on the element's
  free nodes, i.e. the local problem with zero Dirichlet data outside.
* A_e is replaced by its fast-diagonalisation (FDM) approximation
      A~_e = h1 (B~_t (x) B~_s (x) K~_r + B~_t (x) K~_s (x) B~_r + K~_t (x) B~_s (x) B~_r)
             + h2 B~_t (x) B~_s (x) B~_r
  from 1D operators per reference direction: with the element's mean length l
  along that direction, K = (2/l) D^T W D and B = (l/2) W on its n GLL
  points; at an end shared with a neighbour whose mean length normal to the
  shared face is l', the neighbour's end entries are added, K[end,end] +=
  (2/l') (D^T W D)[N,N], B[end,end] += (l'/2) w_N; an end on a Dirichlet face
  is decoupled (its off-diagonal entries in K removed; its value is zero).
  With K S = B S Lambda, S^T B S = I,
      A~_e^{-1} = (S_t (x) S_s (x) S_r) (h1 (L_t + L_s + L_r) + h2)^{-1} (S_t (x) S_s (x) S_r)^T.
  On an axis-aligned affine box the assembled operator is a sum of Kronecker
  products of assembled 1D operators, so A~_e = A_e exactly there.
* Coarse space: the trilinear (N = 1) functions of the element vertices,
  interpolated to the GLL nodes (R_0^T); A_0 = R_0 A R_0^T (Galerkin) on the
  vertices that are not Dirichlet, solved densely here (the paper's XXT is a
  factorisation of the same matrix).
* M^{-1} r = R_0^T A_0^{-1} R_0 r + mask QQ^T (W A~_e^{-1} (W r_e) for every e), where
  r_e is the element's copy of the continuous r and W = mult^{-1/2} at each
  local point: the symmetric form of weighted additive Schwarz (each shared
  node's corrections carry total weight sum_e W^2 = 1).  Measured with this
  oracle on small boxes and pipes (N = 4, random right-hand sides): 22-41
  iterations against 91-207 for Jacobi; without W, 36-70.
"""

import numpy as np
from scipy.linalg import eigh

from . import gll

FACE_AXIS = (0, 0, 1, 1, 2, 2)  # face 2a, 2a+1: the ends of reference direction a (r, s, t)


def element_lengths(mesh):
    """[E, 3] mean length of each element along r, s, t: the mean over the
    n^2 GLL lines in that direction of the distance between their two ends."""
    x = mesh.xyz  # [E, 3, k, j, i]
    lr = np.linalg.norm(x[..., -1] - x[..., 0], axis=1).mean(axis=(1, 2))
    ls = np.linalg.norm(x[..., -1, :] - x[..., 0, :], axis=1).mean(axis=(1, 2))
    lt = np.linalg.norm(x[:, :, -1] - x[:, :, 0], axis=1).mean(axis=(1, 2))
    return np.stack([lr, ls, lt], axis=1)


def face_corner_indices(n, f):
    """(k, j, i) of the four corner GLL nodes of face f of an element."""
    N, end, a = n - 1, (0 if f % 2 == 0 else n - 1), FACE_AXIS[f]
    out = []
    for u in (0, N):
        for v in (0, N):
            out.append((end, v, u) if a == 2 else ((v, end, u) if a == 1 else (v, u, end)))
    return out


def face_neighbours(prob):
    """[E, 6] (element, face) across each face, (-1, -1) on the domain
    boundary.  Two element faces are the same face when they have the same
    four vertices: the global ids of their corner nodes, as a set (so the two
    elements may have any relative orientation)."""
    mesh = prob.mesh
    glo = prob.glo.reshape(prob.shape)
    owner = {}
    for e in range(mesh.E):
        for f in range(6):
            key = tuple(sorted(int(glo[(e,) + c]) for c in face_corner_indices(mesh.n, f)))
            owner.setdefault(key, []).append((e, f))
    nb = -np.ones((mesh.E, 6, 2), dtype=np.int64)
    for pairs in owner.values():
        if len(pairs) == 2:
            (e1, f1), (e2, f2) = pairs
            nb[e1, f1] = (e2, f2)
            nb[e2, f2] = (e1, f1)
    return nb


def fdm_1d(N, l, l_lo, l_hi, dir_lo, dir_hi):
    """(S [n, n], lam [n]) of the 1D pair (K, B) described in the module
    docstring.  l_lo / l_hi: neighbour lengths at the low / high end (None if
    no neighbour); dir_lo / dir_hi: that end is on a Dirichlet face."""
    xi, w = gll.nodes_weights(N)
    D = gll.derivative_matrix(N, xi)
    Kref = D.T @ np.diag(w) @ D
    K = (2.0 / l) * Kref
    B = np.diag((l / 2.0) * w)
    for end, ln, dirichlet in ((0, l_lo, dir_lo), (N, l_hi, dir_hi)):
        if dirichlet:
            d = K[end, end]
            K[end, :] = 0.0
            K[:, end] = 0.0
            K[end, end] = d
        elif ln is not None:
            K[end, end] += (2.0 / ln) * Kref[N, N]
            B[end, end] += (ln / 2.0) * w[N]
    lam, S = eigh(K, B)  # K S = B S diag(lam), S^T B S = I
    return S, lam


class Schwarz:
    """The preconditioner of Eq. 6 for one ``solver.Problem`` (with scalar
    h1, h2); coarse=False keeps the local solves only."""

    def __init__(self, prob, coarse=True):
        if np.ndim(prob.h1) or np.ndim(prob.h2):
            raise ValueError("the separable local solves take scalar h1, h2")
        self.prob = prob
        mesh = prob.mesh
        N, E = mesh.N, mesh.E
        L = element_lengths(mesh)
        nb = face_neighbours(prob)
        self.S = np.empty((E, 3, N + 1, N + 1))
        self.lam = np.empty((E, 3, N + 1))
        for e in range(E):
            for a in range(3):
                ends = []
                for f in (2 * a, 2 * a + 1):
                    e2, f2 = nb[e, f]
                    ln = L[e2, FACE_AXIS[f2]] if e2 >= 0 else None
                    ends.append((ln, bool(mesh.dirichlet_face[e, f])))
                self.S[e, a], self.lam[e, a] = fdm_1d(N, L[e, a], ends[0][0], ends[1][0], ends[0][1], ends[1][1])
        self.coarse = self._coarse_space() if coarse else None

    # -- local solves ------------------------------------------------------
    def local_solve(self, r):
        """A~_e^{-1} applied to each element's local field r[e, k, j, i]."""
        h1, h2 = float(self.prob.h1), float(self.prob.h2)
        Sr, Ss, St = self.S[:, 0], self.S[:, 1], self.S[:, 2]
        v = np.einsum("eli,emj,enk,enml->ekji", Sr, Ss, St, r)  # (S^T (x) S^T (x) S^T) r
        lr, ls, lt = self.lam[:, 0], self.lam[:, 1], self.lam[:, 2]
        den = h1 * (lr[:, None, None, :] + ls[:, None, :, None] + lt[:, :, None, None]) + h2
        v = v / den
        return np.einsum("eli,emj,enk,ekji->enml", Sr, Ss, St, v)  # (S (x) S (x) S) v

    # -- coarse grid -------------------------------------------------------
    def _coarse_space(self):
        """Trilinear vertex functions at the GLL nodes: phi [8, n, n, n], the
        global ids of each element's vertices, the free coarse unknowns and
        the dense A_0 = R_0 A R_0^T on them."""
        prob = self.prob
        N, n = prob.mesh.N, prob.mesh.n
        xi, _ = gll.nodes_weights(N)
        lo, hi = (1 - xi) / 2, (1 + xi) / 2
        phi = np.empty((8, n, n, n))
        corners = []
        for v in range(8):
            bi, bj, bk = v & 1, (v >> 1) & 1, (v >> 2) & 1
            fi, fj, fk = (hi if bi else lo), (hi if bj else lo), (hi if bk else lo)
            phi[v] = fk[:, None, None] * fj[None, :, None] * fi[None, None, :]
            corners.append((N * bk, N * bj, N * bi))
        glo = prob.glo.reshape(prob.shape)
        vid = np.stack([glo[(slice(None),) + c] for c in corners], axis=1)  # [E, 8] global node ids
        mask = prob.mask.reshape(-1)
        first = {}
        for l, g in enumerate(prob.glo):
            first.setdefault(int(g), l)
        free = np.array(sorted({int(g) for g in vid.reshape(-1) if mask[first[int(g)]] > 0}), dtype=np.int64)
        col = {int(g): c for c, g in enumerate(free)}
        cidx = np.array([[col.get(int(g), -1) for g in row] for row in vid])
        self._phi, self._cidx, self._nc = phi, cidx, free.size
        A0 = np.zeros((free.size, free.size))
        for c in range(free.size):
            u = np.zeros(free.size)
            u[c] = 1.0
            A0[:, c] = self.restrict(prob.A(self.prolong(u)))
        return A0

    def prolong(self, c):
        """R_0^T c: the continuous trilinear field of vertex values c, masked."""
        cv = np.where(self._cidx >= 0, c[np.maximum(self._cidx, 0)], 0.0)  # [E, 8]
        u = np.einsum("ev,vkji->ekji", cv, self._phi)
        return self.prob.mask * u

    def restrict(self, r):
        """R_0 r for a continuous r (local copies): each global node counted once."""
        w = np.einsum("ekji,vkji->ev", r / self.prob.mult, self._phi)
        out = np.zeros(self._nc)
        ok = self._cidx >= 0
        np.add.at(out, self._cidx[ok], w[ok])
        return out

    # -- the preconditioner --------------------------------------------------
    def apply(self, r):
        W = self.prob.mult ** -0.5
        z = self.prob.mask * self.prob.gs(W * self.local_solve(W * r))
        if self.coarse is not None and self._nc:
            z = z + self.prolong(np.linalg.solve(self.coarse, self.restrict(r)))
        return z


def pcg(prob, b, precond, tol=1e-10, maxit=20000):
    """PCG as ``solver.pcg`` with z = precond(r) in place of Jacobi."""
    from .solver import BREAKDOWN, CONVERGED, NOT_CONVERGED, Result
    x = np.zeros(prob.shape)
    r = b.copy()
    bnorm = np.sqrt(prob.dot(b, b))
    if bnorm == 0.0:
        return Result(x, 0, 0.0, CONVERGED, [])
    z = precond(r)
    p = z.copy()
    rho = prob.dot(r, z)
    hist = [1.0]
    for k in range(1, maxit + 1):
        w = prob.A(p)
        sigma = prob.dot(p, w)
        if not sigma > 0.0:
            return Result(x, k, hist[-1], BREAKDOWN, hist)
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * w
        rel = np.sqrt(prob.dot(r, r)) / bnorm
        hist.append(rel)
        if rel <= tol:
            return Result(x, k, rel, CONVERGED, hist)
        z = precond(r)
        rho_new = prob.dot(r, z)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return Result(x, maxit, hist[-1], NOT_CONVERGED, hist)
