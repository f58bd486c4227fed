"""Pins for the oracle's GLL nodes, weights and derivative matrix (Sec. 2)."""

import math
import os

import numpy as np
import pytest

from oracle import gll

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = {}
    env = {"sqrt": math.sqrt}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        N, i, node, weight = line.split()
        rows.setdefault(int(N), []).append((eval(node, env), eval(weight, env)))
    return rows


@pytest.mark.parametrize("N", [2, 3, 4])
def test_closed_form_nodes_weights(N):
    x, w = gll.nodes_weights(N)
    ref = _golden()[N]
    np.testing.assert_allclose(x, [r[0] for r in ref], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [r[1] for r in ref], rtol=1e-14, atol=0)


@pytest.mark.parametrize("N", range(1, 13))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = gll.nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13, (N, m)
    # degree 2N is NOT integrated exactly by N+1 Lobatto points
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_exact_on_polynomials(N):
    x, _ = gll.nodes_weights(N)
    D = gll.derivative_matrix(N, x)
    for m in range(N + 1):
        dp = m * x ** (m - 1) if m > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** m, dp, rtol=0, atol=2e-13 * max(1, N * N))


@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_structure(N):
    D = gll.derivative_matrix(N)
    n = N + 1
    assert np.abs(D.sum(axis=1)).max() < 1e-13 * N * N  # D 1 = 0
    flip = D[::-1, ::-1]
    np.testing.assert_allclose(flip, -D, rtol=0, atol=1e-13 * N * N)  # centro-antisymmetric
    assert D[0, 0] == -N * (N + 1) / 4 and D[n - 1, n - 1] == N * (N + 1) / 4


def test_interior_nodes_are_roots_of_legendre_derivative():
    for N in range(2, 13):
        x, _ = gll.nodes_weights(N)
        coeffs = np.polynomial.legendre.Legendre.basis(N).deriv().convert(kind=np.polynomial.Polynomial)
        roots = np.sort(coeffs.roots().real)
        np.testing.assert_allclose(x[1:-1], roots, rtol=0, atol=1e-12)
