"""CPU checks of the host set-up of the overlapping Schwarz local solves
(Sec. 2, Eq. 6) against the oracle: the 1D fast-diagonalisation pairs
(compared through sign-free products, since eigenvectors are fixed only up to
sign) and the per-element data of whole meshes."""

import os

import numpy as np
import pytest

from oracle import mesh, numbering, schwarz, solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    import paper_2109_03592_gb300 as pkg
    from paper_2109_03592_gb300 import build
    if not os.path.exists(os.path.join(ROOT, "paper_2109_03592_gb300", "libsem.so")):
        build.build()
    pkg.lib()
    return pkg.sem


def _same_pair(S, lam, So, lamo, rtol=1e-11):
    """Equal eigenvalues, and equal S diag(1/(lam + c)) S^T (= (K + c B)^{-1}) for two shifts."""
    assert np.abs(lam - lamo).max() <= rtol * np.abs(lamo).max()
    for c in (1.0, 0.1 * lamo.max()):
        a = S @ np.diag(1.0 / (lam + c)) @ S.T
        b = So @ np.diag(1.0 / (lamo + c)) @ So.T
        assert np.abs(a - b).max() <= rtol * np.abs(b).max()


@pytest.mark.parametrize("N,l,llo,lhi,dlo,dhi", [
    (1, 0.5, None, None, False, False),
    (3, 0.3, 0.7, None, False, True),
    (7, 0.125, 0.2, 0.05, False, False),
    (8, 2.0, None, 1.0, True, False),
    (11, 0.01, 0.03, 0.02, False, False),
])
def test_fdm_1d_matches_oracle(sem, N, l, llo, lhi, dlo, dhi):
    S, lam = sem.schwarz_fdm_1d(N, l, llo, lhi, dlo, dhi)
    So, lamo = schwarz.fdm_1d(N, l, llo, lhi, dlo, dhi)
    _same_pair(S, lam, So, lamo)
    # the generalised eigen-relations themselves: S^T B S = I with B the (diagonal) mass
    Bd = np.linalg.inv(S @ S.T)
    assert np.abs(Bd - np.diag(np.diag(Bd))).max() <= 1e-9 * np.abs(Bd).max()


@pytest.mark.parametrize("maker", [lambda: mesh.box(3, 2, 2, 4, 1.0, 2.0, 3.5),
                                   lambda: mesh.pipe(2, 1, 4, 3, L=2.0),
                                   lambda: mesh.pipe(2, 2, 3, 5, L=1.5, periodic=False)])
def test_setup_matches_oracle_element_by_element(sem, maker):
    m_ = maker()
    prob = solver.Problem(m_)
    sw = schwarz.Schwarz(prob, coarse=False)
    glo, _ = numbering.global_numbering(m_)
    S, lam, distinct = sem.schwarz_setup_host(m_.N, glo, m_.xyz, m_.dirichlet_face)
    for e in range(m_.E):
        for a in range(3):
            _same_pair(S[e, a], lam[e, a], sw.S[e, a], sw.lam[e, a])
    assert 1 <= distinct <= 3 * m_.E
    if m_.kind == "pipe" and m_.period is not None:
        # every layer of a periodic pipe is the same: at most 3 problems per cross-section element
        n2d = m_.E // 4
        assert distinct <= 3 * n2d


def test_setup_rejects_invalid_input(sem):
    with pytest.raises(sem.SemError) as ei:
        sem.schwarz_fdm_1d(3, -1.0)
    assert ei.value.status == sem.SEM_ERR_INVALID
    m_ = mesh.box(1, 1, 1, 1)
    glo, _ = numbering.global_numbering(m_)
    with pytest.raises(sem.SemError) as ei:
        sem.schwarz_setup_host(1, glo, m_.xyz, m_.dirichlet_face)
    assert ei.value.status == sem.SEM_ERR_INVALID
