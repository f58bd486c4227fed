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
        sem.schwarz_setup_host(12, glo, m_.xyz, m_.dirichlet_face)  # orders above 11 are not compiled
    assert ei.value.status == sem.SEM_ERR_INVALID


def flipped_pair(N):
    """Two elements sharing the face x = 1: element 0 is [0, 1]^3 with local
    axes along x, y, z; element 1 is [1, 2.5] x [0, 1] x [0, 1] turned half a
    turn about the x axis (local s along -y, t along -z, still right-handed).
    The shared face is i = N of element 0 and i = 0 of element 1, with its two
    in-face directions reversed between them.  Every other face is Dirichlet."""
    xi, _ = mesh.gll.nodes_weights(N)
    n = N + 1
    u = (1.0 + xi) / 2
    xyz = np.empty((2, 3, n, n, n))
    xyz[0, 0] = u[None, None, :]
    xyz[0, 1] = u[None, :, None]
    xyz[0, 2] = u[:, None, None]
    xyz[1, 0] = (1.0 + 1.5 * u)[None, None, :]
    xyz[1, 1] = (1.0 - u)[None, :, None]
    xyz[1, 2] = (1.0 - u)[:, None, None]
    dface = np.ones((2, 6), dtype=bool)
    dface[0, 1] = dface[1, 0] = False
    return mesh.Mesh(N, xyz, dface)


@pytest.mark.parametrize("N", [3, 4, 7])
def test_faces_match_by_their_vertices_in_any_orientation(sem, N):
    """The face-neighbour rule pairs two faces with the same four vertices
    whatever the elements' relative orientation.  At odd N the centre-most
    face node of one element is not that of the other here (reversed in-face
    directions), so a rule through that node would miss the pair and drop the
    neighbour's end entries; the oracle and the host set-up must both find it
    (element 1 is longer, so the neighbour's length changes element 0's r
    operator)."""
    m_ = flipped_pair(N)
    prob = solver.Problem(m_)
    nb = schwarz.face_neighbours(prob)
    assert tuple(nb[0, 1]) == (1, 0) and tuple(nb[1, 0]) == (0, 1)
    assert (nb[0, [0, 2, 3, 4, 5]] == -1).all() and (nb[1, 1:] == -1).all()
    sw = schwarz.Schwarz(prob, coarse=False)
    # element 0's r operator: Dirichlet at i = 0, the neighbour's length 1.5 at i = N
    _same_pair(sw.S[0, 0], sw.lam[0, 0], *schwarz.fdm_1d(N, 1.0, None, 1.5, True, False))
    alone = schwarz.fdm_1d(N, 1.0, None, None, True, False)  # the same end with no neighbour found
    assert not np.allclose(sw.lam[0, 0], alone[1])
    S, lam, _ = sem.schwarz_setup_host(N, prob.glo, m_.xyz, m_.dirichlet_face)
    for e in range(2):
        for a in range(3):
            _same_pair(S[e, a], lam[e, a], sw.S[e, a], sw.lam[e, a])
