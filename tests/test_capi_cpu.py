"""The C-ABI library loads and exports every entry point include/aica.h
declares; host-side argument and mesh validation (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_cs_0702131_gb300 import build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    from paper_cs_0702131_gb300 import aica
    return aica.lib()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "aica.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(aica_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    from paper_cs_0702131_gb300 import aica
    assert names == set(aica.SIGNATURES)


def test_null_arguments(L):
    out = ctypes.c_void_p()
    assert L.aica_mesh_create(None, 0, None, None, 0, None, None, 0, None, ctypes.byref(out)) == 1
    assert b"NULL" in L.aica_last_error()
    assert L.aica_build_interaction_list(None, 2.5, 0.0, None) == 1
    assert L.aica_bin_molecules(None, None, None, 0, None, None, None, None) == 1
    assert L.aica_forces(None, None, 0, None, None, None, None) == 1
    assert L.aica_forces_backward(None, None, 0, None, None, None, None, None) == 1
    assert L.aica_status_string(3) == b"AICA_ERR_OUTSIDE_MESH"
    assert L.aica_last_launch_count(None) == 0


def _create(L, mesh, box):
    from paper_cs_0702131_gb300 import aica
    try:
        h = aica.aica_mesh_create(mesh["points"], mesh["face_offsets"], mesh["face_vertices"], mesh["owner"],
                                  mesh["neighbour"], mesh["n_cells"], box["L"], box["periodic"])
    except aica.AicaError as e:
        return e.name
    aica.aica_mesh_destroy(h)
    return "AICA_OK"


def test_bad_meshes_rejected_on_host(L):
    pts, cells = synth.cube_cells([(0, 0, 0), (2, 0, 0)])
    box = dict(L=np.array([10.0, 10, 10]), periodic=np.array([0, 0, 0], np.int32))
    good = synth.cells_to_mesh(pts, cells)
    # an open cell: drop one face
    open_ = dict(good, face_offsets=good["face_offsets"][:-1], face_vertices=good["face_vertices"][:-4],
                 owner=good["owner"][:-1], neighbour=good["neighbour"][:-1])
    assert _create(L, open_, box) == "AICA_ERR_BAD_MESH"
    # an inverted cell: every face of cell 0 reversed
    fv = good["face_vertices"].reshape(-1, 4).copy()
    fv[good["owner"] == 0] = fv[good["owner"] == 0][:, ::-1]
    inv = dict(good, face_vertices=fv.reshape(-1))
    assert _create(L, inv, box) == "AICA_ERR_BAD_MESH"
    # a vertex index out of range
    bad = dict(good, face_vertices=np.where(good["face_vertices"] == 3, 99, good["face_vertices"]))
    assert _create(L, bad, box) == "AICA_ERR_BAD_MESH"
    # a cell outside its periodic box
    box_p = dict(L=np.array([2.5, 10, 10]), periodic=np.array([1, 0, 0], np.int32))
    assert _create(L, good, box_p) == "AICA_ERR_BAD_MESH"


def test_coupling_transform_on_host(L):
    """aica_coupling_transform (host arithmetic, §2.2.2) against the oracle's
    own construction; antiparallel normals give R = I, parallel ones are
    rejected."""
    from oracle import transforms as T
    from paper_cs_0702131_gb300.aica import AicaError, aica_coupling_transform
    rng = np.random.default_rng(12)
    for _ in range(25):
        na, nb = rng.normal(size=3), rng.normal(size=3)
        ca, cb = rng.normal(size=3) * 5, rng.normal(size=3) * 5
        R, y = aica_coupling_transform(na, ca, nb, cb)
        Ro, yo = T.coupling(na, ca, nb, cb)
        np.testing.assert_allclose(R, Ro, atol=1e-13)
        np.testing.assert_allclose(y, yo, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        np.testing.assert_allclose(R @ (-na / np.linalg.norm(na)), nb / np.linalg.norm(nb), atol=1e-13)
    R, y = aica_coupling_transform(np.array([1.0, 0, 0]), np.array([3.0, 0, 0]), np.array([-1.0, 0, 0]),
                                   np.array([0.0, 0, 0]))
    np.testing.assert_array_equal(R, np.eye(3))
    np.testing.assert_allclose(y, [-3.0, 0, 0])
    with pytest.raises(AicaError) as e:
        aica_coupling_transform(np.array([0.0, 0, 1]), np.zeros(3), np.array([0.0, 0, 2]), np.zeros(3))
    assert e.value.name == "AICA_ERR_INVALID_ARG"
