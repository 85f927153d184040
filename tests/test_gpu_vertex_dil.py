"""The paper's vertex-vertex list criterion (§2.2, App. A.1) on the GPU:
lists bit-exact against the oracle's vertex mode, forces equal to the §2.3
loops over those lists, and the twisted-mesh miss of §2.2."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import Mesh, aica_get_list_info
from gpu_helpers import compare_lists

pytestmark = pytest.mark.gpu


def _setup(c, criterion, skin=None):
    m = Mesh(c["mesh"], c["box"])
    m.build_lists(c["rc"], c["skin"] if skin is None else skin, criterion=criterion)
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    m.bin(pos, sp)
    return m


@pytest.mark.parametrize("name,seed", [("t0", 0), ("h0", 1), ("c1", 2)])
def test_vertex_lists_and_forces_equal_oracle(name, seed):
    c = synth.make(name, seed)
    m = _setup(c, "vertex")
    assert aica_get_list_info(m.h).criterion == 1
    geo = oracle.cell_geometry(c["mesh"])
    o = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo, criterion="vertex")
    g = m.lists()
    assert g["ties"] == 0 and o["ties"] == 0
    compare_lists(g, o)
    cell, wrapped = oracle.locate(geo, c["box"], c["pos"])
    order, off = oracle.bin_order(cell, geo["n_cells"])
    loop = oracle.aica_loop(o, off, wrapped[order], c["species"][order], c["eps"], c["sigma"], c["rc"], c["box"])
    Fo = np.empty_like(loop["F"])
    Fo[order] = loop["F"]
    ref = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    scale = ref["Fabs"][:, None]
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        F, ev, counts = m.forces(c["eps"], c["sigma"], prec)
        assert np.abs(F.double().cpu().numpy() - Fo).max() / scale.max() <= tol
        cnt = counts.cpu().numpy()
        assert list(cnt[3:5]) == list(loop["counts"][3:5]) and 2 * cnt[5] == loop["counts"][5]
        assert abs(ev[0].item() - loop["U"]) <= 1e-6 * ref["Uabs"]
    m.close()


def test_vertex_lists_are_a_subset_on_tets():
    c = synth.make("t0", 4)
    mv, mm = _setup(c, "vertex"), _setup(c, "min_distance")
    gv, gm = mv.lists(), mm.lists()
    assert len(gv["dil_ids"]) < len(gm["dil_ids"])
    for i in range(c["mesh"]["n_cells"]):
        a = set(gv["dil_ids"][gv["dil_off"][i]:gv["dil_off"][i + 1]].tolist())
        b = set(gm["dil_ids"][gm["dil_off"][i]:gm["dil_off"][i + 1]].tolist())
        assert a <= b
    mv.close(); mm.close()


def test_twisted_cells_missed_by_vertex_rule():
    """Two tetrahedra whose long edges cross 1.0 apart, every vertex pair
    farther than 3.8: one pair of molecules 1.2 apart across the crossing."""
    pts = np.array([[-3, 0, 0], [3, 0, 0], [0, -0.5, -2], [0, 0.5, -2],
                    [0, -3, 1], [0, 3, 1], [-0.5, 0, 3], [0.5, 0, 3]], float) + 10.0
    mesh = synth.cells_to_mesh(pts, np.array([[0, 1, 2, 3], [4, 5, 6, 7]]))
    box = dict(L=np.array([100.0, 100.0, 100.0]), periodic=np.array([0, 0, 0], np.int32))
    c = dict(mesh=mesh, box=box, rc=2.5, skin=0.0, pos=np.array([[10.0, 10.0, 9.9], [10.0, 10.0, 11.1]]),
             species=np.zeros(2, np.int32), eps=np.array([1.0]), sigma=np.array([1.0]))
    for criterion, within in (("vertex", 0), ("min_distance", 1)):
        m = _setup(c, criterion)
        F, ev, counts = m.forces(c["eps"], c["sigma"], "fp64")
        assert int(counts[4].item()) == within
        if within == 0:
            assert float(F.abs().max()) == 0.0
        m.close()
