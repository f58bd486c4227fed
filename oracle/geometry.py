"""Geometric factors g1..g6 and the diagonal mass B.

Test infrastructure only (see ``oracle/__init__``).

Alg. 1 contracts the reference-space gradient (rtmp, stmp, ttmp) with six
per-point factors g1xyz..g6xyz: wr uses (g1, g4, g5), ws uses (g4, g2, g6)
and wt uses (g5, g6, g3), i.e. a symmetric 3x3 matrix
G = [[g1, g4, g5], [g4, g2, g6], [g5, g6, g3]].  The paper uses G without
defining it; the reading taken here is the standard isoparametric one:

    J_ab   = d x_a / d r_b         (D applied to the nodal coordinates)
    G      = w_i w_j w_k det(J) J^{-1} J^{-T}
    B      = w_i w_j w_k det(J)    (the GLL-quadrature mass of Sec. 2, Eq. 4)

so that u^T (stiffness) v = sum_q grad_r u . G grad_r v approximates
int grad u . grad v dx.
"""

import numpy as np

from . import gll


def reference_gradient(D, f):
    """(d f/dr, d f/ds, d f/dt) of an element-local field f[e, k, j, i]:
    f_r = sum_l D_il f_ljk, f_s = sum_l D_jl f_ilk, f_t = sum_l D_kl f_ijl."""
    fr = np.einsum("il,ekjl->ekji", D, f)
    fs = np.einsum("jl,ekli->ekji", D, f)
    ft = np.einsum("kl,elji->ekji", D, f)
    return fr, fs, ft


def jacobian(mesh):
    """J[e, k, j, i, a, b] = d x_a / d r_b at every GLL point.

    D applied to the coordinates relative to the element's first node: D
    annihilates constants, so this is the same J, without the O(|x|/h)
    cancellation that absolute coordinates cause for small elements far
    from the origin."""
    D = gll.derivative_matrix(mesh.N)
    E, n = mesh.E, mesh.n
    J = np.empty((E, n, n, n, 3, 3))
    for a in range(3):
        x = mesh.xyz[:, a] - mesh.xyz[:, a, :1, :1, :1]
        fr, fs, ft = reference_gradient(D, x)
        J[..., a, 0] = fr
        J[..., a, 1] = fs
        J[..., a, 2] = ft
    return J


def factors(mesh):
    """Return (G [E, 6, n, n, n] ordered g1..g6, B [E, n, n, n], detJ).

    Raises ValueError when some det(J) <= 0 (an inverted element)."""
    _, w = gll.nodes_weights(mesh.N)
    J = jacobian(mesh)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("mesh has an element with det(J) <= 0")
    Jinv = np.linalg.inv(J)  # Jinv[..., b, a] = d r_b / d x_a
    M = np.einsum("...ba,...ca->...bc", Jinv, Jinv)  # J^{-1} J^{-T}
    w3 = w[:, None, None] * w[None, :, None] * w[None, None, :]  # [k, j, i]
    scale = w3[None] * detJ
    G = np.empty((mesh.E, 6, mesh.n, mesh.n, mesh.n))
    G[:, 0] = scale * M[..., 0, 0]  # g1 = G_rr
    G[:, 1] = scale * M[..., 1, 1]  # g2 = G_ss
    G[:, 2] = scale * M[..., 2, 2]  # g3 = G_tt
    G[:, 3] = scale * M[..., 0, 1]  # g4 = G_rs
    G[:, 4] = scale * M[..., 0, 2]  # g5 = G_rt
    G[:, 5] = scale * M[..., 1, 2]  # g6 = G_st
    B = scale.copy()
    return G, B, detJ
