"""Edge cases of the CUDA path against the oracle: no molecules, one
molecule, empty cells, a crowded cell (more molecules than a chunk, a lane
group or a warp), pairs exactly at and just inside the cut-off."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import Mesh

pytestmark = pytest.mark.gpu

L = 12.0
BOX = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
EPS, SIG = np.array([1.0]), np.array([1.0])


def _mesh(tets):
    return synth.hex_mesh((4, 4, 4), (0, 0, 0), (L, L, L), 0.1, np.random.default_rng(3), tets=tets)


def _forces(mesh, pos, prec, rc=2.5):
    m = Mesh(mesh, BOX)
    m.build_lists(rc, 1e-3)
    p = torch.tensor(np.asarray(pos, float).reshape(-1, 3), dtype=torch.float64, device="cuda")
    sp = torch.zeros(p.shape[0], dtype=torch.int32, device="cuda")
    m.bin(p, sp)
    F, ev, cnt = m.forces(EPS, SIG, prec)
    out = F.double().cpu().numpy(), ev.cpu().numpy(), cnt.cpu().numpy()
    m.close()
    return out


@pytest.mark.parametrize("tets", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_no_molecules_and_one_molecule(tets, prec):
    F, ev, cnt = _forces(_mesh(tets), np.zeros((0, 3)), prec)
    assert F.shape == (0, 3) and np.all(ev == 0) and np.all(cnt == 0)
    F, ev, cnt = _forces(_mesh(tets), [[5.0, 5.0, 5.0]], prec)
    assert np.all(F == 0) and np.all(ev == 0) and np.all(cnt == 0)


def _check(pos, prec, tets, rc=2.5):
    pos = np.asarray(pos, float)
    F, ev, cnt = _forces(_mesh(tets), pos, prec, rc)
    ref = oracle.lj(pos, np.zeros(len(pos), np.int32), EPS, SIG, rc, BOX)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(F - ref["F"]).max() <= tol * max(ref["Fabs"].max(), 1e-300)
    assert cnt[3] + cnt[4] + cnt[5] == ref["pairs"]
    assert abs(ev[0] - ref["U"]) <= (1e-12 if prec == "fp64" else 1e-6) * max(ref["Uabs"], 1e-300)


@pytest.mark.parametrize("tets", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_mostly_empty_cells(tets, prec):
    rng = np.random.default_rng(7)
    _check(rng.uniform(0, L, size=(9, 3)), prec, tets)


@pytest.mark.parametrize("tets", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_crowded_cell(tets, prec):
    """70 molecules in one small region (several chunks, more than a lane
    group and a warp in one cell), plus a dilute background."""
    rng = np.random.default_rng(11)
    g = np.stack(np.meshgrid(*[np.arange(5) * 0.9] * 3, indexing="ij"), -1).reshape(-1, 3)[:70]
    crowd = 4.3 + g * 0.35 + rng.normal(scale=0.01, size=g.shape)
    back = rng.uniform(0, L, size=(40, 3))
    _check(np.concatenate([crowd, back]), prec, tets)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pairs_at_and_just_inside_the_cut(prec):
    """r = rc exactly is out (strict), r = rc - 1e-9 is in: FP32 cannot tell
    them apart, the FP64 re-decision near the cut does."""
    pos = [[2.0, 2.0, 2.0], [4.5, 2.0, 2.0],          # r = 2.5 exactly
           [2.0, 8.0, 2.0], [4.5 - 1e-9, 8.0, 2.0],   # just inside
           [8.0, 8.0, 8.0], [8.0, 8.0, 10.5 + 1e-9]]  # just outside
    F, ev, cnt = _forces(_mesh(True), pos, prec)
    assert cnt[3] + cnt[4] + cnt[5] == 1
    assert np.all(F[[0, 1, 4, 5]] == 0) and np.all(F[[2, 3], 0] != 0)
    _check(pos, prec, True)


@pytest.mark.parametrize("tets", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_clusters_larger_than_the_survivor_buffer(tets, prec):
    """A liquid at rho* = 0.8 in 2^3 hexahedra of about 6 sigma (about 171
    molecules per hexahedron, the FP32 kernel's cluster): a cluster's own
    molecules no longer fit the survivor buffer's fill threshold, so the
    buffer is evaluated in the middle of pushing them, over many tiles.
    Every molecule at the stated tolerance, energy, virial and pair counts
    against the oracle."""
    from gpu_helpers import assert_forces
    a = (4 / 0.8) ** (1 / 3)
    n = 7
    Lb = n * a
    box = dict(L=np.array([Lb, Lb, Lb]), periodic=np.array([1, 1, 1], np.int32))
    rng = np.random.default_rng(21)
    pos = synth.wrap(synth.fcc_sites(n, n, n, a) + rng.normal(scale=0.05, size=(4 * n ** 3, 3)), box["L"],
                     box["periodic"])
    mesh = synth.hex_mesh((2, 2, 2), (0, 0, 0), (Lb, Lb, Lb), 0.1, np.random.default_rng(4), tets=tets)
    m = Mesh(mesh, box)
    m.build_lists(2.5, 1e-3)
    assert m.get_option("cluster_path") == 1
    p = torch.tensor(pos, dtype=torch.float64, device="cuda")
    sp = torch.zeros(len(pos), dtype=torch.int32, device="cuda")
    m.bin(p, sp)
    F, ev, cnt = m.forces(EPS, SIG, prec)
    ref = oracle.lj(pos, np.zeros(len(pos), np.int32), EPS, SIG, 2.5, box)
    assert_forces(F.double().cpu().numpy(), ref, 1e-12 if prec == "fp64" else 1e-5)
    ev = ev.cpu().numpy()
    cnt = cnt.cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(ev[0] - ref["U"]) <= tol * ref["Uabs"]
    np.testing.assert_allclose(ev[1:7], ref["W"], rtol=0, atol=tol * ref["Wabs"])
    assert cnt[3] + cnt[4] + cnt[5] == ref["pairs"]
    m.close()
