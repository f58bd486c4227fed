"""GLL nodes, quadrature weights and the Lagrange derivative matrix D.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2 of the paper: each element carries a tensor product of 1D Lagrange
interpolants of order N on the Gauss-Lobatto-Legendre (GLL) points; Alg. 1
applies their derivative matrix (``dxm1``) and its transpose (``dxtm1``).
The constructions below are the textbook ones (Canuto, Hussaini,
Quarteroni & Zang, "Spectral Methods", Sec. 2.3; Deville, Fischer & Mund,
"High-Order Methods for Incompressible Fluid Flow", Sec. 2.4).
"""

import numpy as np


def legendre(N, x):
    """Return (P_N(x), P_{N-1}(x)) by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, P_0 = 1, P_1 = x."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, N):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        p_prev, p = p, p_next
    return p, p_prev


def nodes_weights(N):
    """GLL nodes xi_0 < ... < xi_N and weights w_i = 2 / (N(N+1) P_N(xi_i)^2).

    The nodes are -1, +1 and the roots of P_N'.  They are the zeros of
    f(x) = (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)); the Legendre
    equation gives f'(x) = -N(N+1) P_N(x), so Newton's step is
    x <- x - (x P_N - P_{N-1}) / ((N+1) P_N), started from the
    Chebyshev-Gauss-Lobatto points -cos(pi i / N).
    """
    if N < 1:
        raise ValueError("GLL needs N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(100):
        pn, pn1 = legendre(N, x)
        dx = (x * pn - pn1) / ((N + 1) * pn)
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    x = np.sort(x)
    pn, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pn * pn)
    return x, w


def derivative_matrix(N, x=None):
    """D_ij = l_j'(xi_i) for the GLL Lagrange basis (closed form):
    D_ij = P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j)) for i != j,
    D_00 = -N(N+1)/4, D_NN = +N(N+1)/4, D_ii = 0 otherwise."""
    if x is None:
        x, _ = nodes_weights(N)
    pn, _ = legendre(N, x)
    n = N + 1
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = pn[i] / (pn[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def lagrange_eval(x_nodes, j, t):
    """Value of the j-th Lagrange cardinal polynomial on x_nodes at t (used by
    tests to evaluate fields between nodes)."""
    v = np.ones_like(np.asarray(t, dtype=np.float64))
    for m, xm in enumerate(x_nodes):
        if m != j:
            v = v * (t - xm) / (x_nodes[j] - xm)
    return v
