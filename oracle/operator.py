"""The matrix-free local SEM operator (Alg. 1 plus the Helmholtz mass term).

Test infrastructure only (see ``oracle/__init__``).

Alg. 1 (CUDA Fortran ``axhelm``) computes, per element and GLL point (i,j,k):

    rtmp = sum_l D_il u_ljk,  stmp = sum_l D_jl u_ilk,  ttmp = sum_l D_kl u_ijl
    (wr, ws, wt) = h1 * G (rtmp, stmp, ttmp)        G from g1..g6 (geometry.py)
    w_ijk = sum_l [ D_li wr_ljk + D_lj ws_ilk + D_lk wt_ijl ]

(``shdxtm1(i,l)`` is D transposed, so its (i,l) entry is D_li.)  The listing
elides the rest of the subroutine; Sec. 2, Eq. 4 solves
(b0/dt - Re^{-1} grad^2) u = ..., whose discrete form is h1 * stiffness +
h2 * mass.  The reading taken here adds h2 * B_ijk * u_ijk to w.  Alg. 1
reads h1 per local point, h1(i,j,k,e); h1 and h2 here are either scalars (one
value per solve) or arrays shaped like u, one value per local point, with h2
per point read the same way (a variable mass coefficient).
"""

import numpy as np

from . import gll
from .geometry import reference_gradient


def ax_local(u, G, B, D, h1=1.0, h2=0.0):
    """w = A_L u on element-local fields u[e, k, j, i] (no assembly, no mask).
    h1, h2: scalars or arrays [e, k, j, i] (per local point)."""
    ur, us, ut = reference_gradient(D, u)
    g1, g2, g3, g4, g5, g6 = (G[:, c] for c in range(6))
    wr = h1 * (g1 * ur + g4 * us + g5 * ut)
    ws = h1 * (g4 * ur + g2 * us + g6 * ut)
    wt = h1 * (g5 * ur + g6 * us + g3 * ut)
    w = (np.einsum("li,ekjl->ekji", D, wr)
         + np.einsum("lj,ekli->ekji", D, ws)
         + np.einsum("lk,elji->ekji", D, wt))
    if np.any(h2 != 0.0):
        w = w + h2 * B * u
    return w


def local_diagonal(G, B, D, h1=1.0, h2=0.0):
    """Diagonal of A_L, element by element.  With Gh = h1 G (h1 taken at each
    point where G is):

    diag_ijk = sum_l D_li^2 Gh1_ljk + sum_l D_lj^2 Gh2_ilk + sum_l D_lk^2 Gh3_ijl
               + 2 D_ii D_jj Gh4_ijk + 2 D_ii D_kk Gh5_ijk + 2 D_jj D_kk Gh6_ijk
               + h2_ijk B_ijk

    (substituting u = e_ijk into ax_local: ur at point (l,j,k) is D_li, and
    wr there is scaled by h1 at (l,j,k); the cross terms survive only where
    both one-dimensional derivatives sit on the point itself).  A scalar h1
    factors out of the whole bracket."""
    D2 = D * D
    dd = np.diag(D)
    h1 = np.asarray(h1, dtype=np.float64)
    if h1.ndim:
        G = G * h1[:, None]
    g1, g2, g3, g4, g5, g6 = (G[:, c] for c in range(6))
    diag = (np.einsum("li,ekjl->ekji", D2, g1)
            + np.einsum("lj,ekli->ekji", D2, g2)
            + np.einsum("lk,elji->ekji", D2, g3))
    di = dd[None, None, None, :]
    dj = dd[None, None, :, None]
    dk = dd[None, :, None, None]
    diag = diag + 2.0 * di * dj * g4 + 2.0 * di * dk * g5 + 2.0 * dj * dk * g6
    if not h1.ndim:
        diag = float(h1) * diag
    return diag + h2 * B


def element_matrix_affine(N, hx, hy, hz, h1=1.0, h2=0.0):
    """Explicit (n^3 x n^3) matrix of A_L on one affine element of size
    hx x hy x hz, built from 1D matrices: with W = diag(w) and K = D^T W D,
    A = h1 [ (hy hz / 2hx) W(x)W(x)K + (hx hz / 2hy) W(x)K(x)W + (hx hy / 2hz) K(x)W(x)W ]
        + h2 (hx hy hz / 8) W(x)W(x)W
    where (x) is the Kronecker product with the k factor leftmost (i fastest).
    Used only as an independent pin for ax_local."""
    x, w = gll.nodes_weights(N)
    D = gll.derivative_matrix(N, x)
    W = np.diag(w)
    K = D.T @ W @ D
    kron3 = lambda a, b, c: np.kron(a, np.kron(b, c))  # noqa: E731  (k, j, i)
    A = h1 * ((hy * hz / (2 * hx)) * kron3(W, W, K)
              + (hx * hz / (2 * hy)) * kron3(W, K, W)
              + (hx * hy / (2 * hz)) * kron3(K, W, W))
    A = A + h2 * (hx * hy * hz / 8.0) * kron3(W, W, W)
    return A
