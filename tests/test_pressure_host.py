"""CPU checks of the host side of the P_N - P_{N-2} pressure space (Sec. 2:
pressure on the Gauss-Legendre points of order N-2): the library's GL nodes,
weights and GLL-basis interpolation/derivative matrices against the oracle,
which builds them another way (numpy's Gauss-Legendre rule, the product rule
for the Lagrange derivative)."""

import os

import numpy as np
import pytest

from oracle import pressure

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    import paper_2109_03592_gb300 as pkg
    from paper_2109_03592_gb300 import build
    if not os.path.exists(os.path.join(ROOT, "paper_2109_03592_gb300", "libsem.so")):
        build.build()
    pkg.lib()
    return pkg.sem


@pytest.mark.parametrize("N", list(range(2, 12)))
def test_gl_basis_matches_oracle(sem, N):
    z, r, Ig, DIg = sem.pressure_basis(N)
    zo, ro = pressure.gl_nodes_weights(N - 1)
    Io, Do, _ = pressure.interpolation_matrices(N)
    np.testing.assert_allclose(z, zo, rtol=0, atol=2e-15)
    np.testing.assert_allclose(r, ro, rtol=0, atol=2e-15)
    assert np.abs(Ig - Io).max() <= 1e-14 * np.abs(Io).max()
    assert np.abs(DIg - Do).max() <= 2e-13 * np.abs(Do).max()
    # partition of unity: the basis interpolates constants exactly, and differentiates them to 0
    np.testing.assert_allclose(Ig.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert np.abs(DIg.sum(axis=1)).max() <= 1e-12 * np.abs(DIg).max()


@pytest.mark.parametrize("N", [1, 12])
def test_gl_basis_rejects_orders_outside_the_pressure_space(sem, N):
    with pytest.raises(sem.SemError) as ei:
        sem.pressure_basis(N)
    assert ei.value.status == sem.SEM_ERR_INVALID
