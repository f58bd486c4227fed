"""CPU checks of the C ABI: the library loads, exports every symbol that
include/sem.h declares, and its host-side topology matches the oracle."""

import os
import re

import numpy as np
import pytest

from oracle import mesh as omesh, numbering

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    import paper_2109_03592_gb300 as pkg
    from paper_2109_03592_gb300 import build
    if not os.path.exists(os.path.join(ROOT, "paper_2109_03592_gb300", "libsem.so")):
        build.build()
    pkg.lib()
    return pkg.sem


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(sem):
    names = declared_functions()
    assert len(names) >= 20
    lib = sem.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in sem.SIGNATURES, name
    assert set(sem.SIGNATURES) == set(names)


def test_status_strings(sem):
    lib = sem.lib()
    assert lib.sem_status_str(0) == b"SEM_OK"
    assert lib.sem_status_str(8) == b"SEM_ERR_BAD_MESH"
    assert lib.sem_version() >= 1


@pytest.mark.parametrize("desc,maker", [
    (dict(kind="box", nx=3, ny=2, nz=2, N=3), lambda: omesh.box(3, 2, 2, 3)),
    (dict(kind="box", nx=1, ny=1, nz=1, N=1), lambda: omesh.box(1, 1, 1, 1)),
    (dict(kind="pipe", nc=2, nr=1, nzp=3, N=3, L=3.0), lambda: omesh.pipe(2, 1, 3, 3, L=3.0)),
    (dict(kind="pipe", nc=4, nr=2, nzp=3, N=2, L=3.0, periodic=False),
     lambda: omesh.pipe(4, 2, 3, 2, L=3.0, periodic=False)),
    (dict(kind="pipe", nc=3, nr=2, nzp=4, N=4, L=2.0), lambda: omesh.pipe(3, 2, 4, 4, L=2.0)),
])
def test_topological_numbering_matches_oracle_bit_exact(sem, desc, maker):
    vert = sem.mesh_vertices(desc)
    glo, ng = sem.topology_numbering(vert.shape[0], desc["N"], vert)
    og, opg = numbering.global_numbering(maker())
    assert ng == opg
    assert np.array_equal(glo, og)


def test_numbering_of_shuffled_vertex_ids(sem):
    # any relabelling of the vertices gives the same node partition
    desc = dict(kind="pipe", nc=2, nr=2, nzp=3, N=3, L=3.0)
    vert = sem.mesh_vertices(desc)
    perm = np.random.default_rng(1).permutation(vert.max() + 1) * 7 + 11
    g1, n1 = sem.topology_numbering(vert.shape[0], 3, vert)
    g2, n2 = sem.topology_numbering(vert.shape[0], 3, perm[vert])
    assert n1 == n2 and np.array_equal(g1, g2)


def test_pipe_node_count_closed_form_large(sem):
    desc = dict(kind="pipe", nc=8, nr=2, nzp=32, N=7)
    vert = sem.mesh_vertices(desc)
    assert vert.shape[0] == 4096
    glo, ng = sem.topology_numbering(4096, 7, vert)
    assert ng == omesh.pipe_global_node_count(8, 2, 32, 7)
    mult = np.bincount(glo)
    assert mult.max() == 8 and np.bincount(mult)[6] > 0
    # first touch
    assert glo[0] == 0 and np.all(np.diff(np.maximum.accumulate(glo)) <= 1)


@pytest.mark.parametrize("bad", [
    dict(kind="box", nx=0, ny=1, nz=1, N=3),
    dict(kind="box", nx=1, ny=1, nz=1, N=12),
    dict(kind="pipe", nc=2, nr=1, nzp=2, N=3),  # periodic pipe needs nzp >= 3
    dict(kind="pipe", nc=2, nr=1, nzp=3, N=3, a=0.9),  # square corner outside the circle
])
def test_invalid_descriptors_rejected(sem, bad):
    with pytest.raises(sem.SemError) as ei:
        sem.mesh_vertices(bad)
    assert ei.value.status == sem.SEM_ERR_INVALID


def test_inconsistent_topology_rejected(sem):
    vert = sem.mesh_vertices(dict(kind="box", nx=2, ny=1, nz=1, N=2))
    vert[1, 3] = vert[1, 2]  # repeated corner id
    with pytest.raises(sem.SemError) as ei:
        sem.topology_numbering(2, 2, vert)
    assert ei.value.status == sem.SEM_ERR_BAD_MESH


# entry points whose first argument is a handle (mesh, space, preconditioner,
# server) or a descriptor; host-only helpers with sizes first are checked
# elsewhere
_HANDLE_CALLS = ("sem_mesh_", "sem_ax", "sem_gs", "sem_rhs", "sem_apply", "sem_jacobi", "sem_pcg_", "sem_proj_",
                 "sem_pressure_", "sem_schwarz_", "sem_server_")
_HOST_ONLY = {"sem_mesh_vertices", "sem_pressure_basis", "sem_schwarz_fdm_1d", "sem_schwarz_setup_host",
              "sem_gs_halo", "sem_topology_numbering"}


def test_every_entry_point_rejects_null_handles_without_a_gpu(sem):
    """Every status-returning call given null handles and buffers returns a
    status and never aborts: SEM_OK for the destroy calls (a null handle is
    nothing to free), SEM_ERR_INVALID otherwise.  No call reaches the GPU."""
    import ctypes as C
    lib = sem.lib()
    checked = 0
    for name, (res, args) in sem.SIGNATURES.items():
        if res is not C.c_int or name in _HOST_ONLY or not name.startswith(_HANDLE_CALLS):
            continue
        if name in ("sem_mesh_fp64_kernel", "sem_mesh_ax_variant"):
            continue  # not a status: -1 or a variant number
        vals = []
        for a in args:
            if a in (C.c_double, C.c_float):
                vals.append(1.0)
            elif a in (C.c_int, C.c_int64, C.c_uint64, C.c_size_t, C.c_uint32, C.c_int32):
                vals.append(1)
            else:
                vals.append(None)
        st = getattr(lib, name)(*vals)
        want = sem.SEM_OK if name.endswith("_destroy") else sem.SEM_ERR_INVALID
        assert st == want, (name, st)
        checked += 1
    assert checked >= 35
