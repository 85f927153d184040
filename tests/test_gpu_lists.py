"""GPU interaction lists against the oracle: bit-exact (§2.2, App. A)."""
import numpy as np
import pytest

import oracle
from paper_cs_0702131_gb300 import synth
from gpu_helpers import compare_lists, gpu_setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,seed", [("t0", 0), ("t0", 5), ("c1", 0), ("h0", 1)])
def test_lists_equal_oracle_full(name, seed):
    c = synth.make(name, seed)
    m, *_ = gpu_setup(c)
    g = m.lists()
    o = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"])
    assert g["ties"] == 0 and o["ties"] == 0
    compare_lists(g, o)


def test_lists_open_axis_and_removed_cells():
    c = synth.nanochannel(2, nfcc=(12, 4, 12), hex_shape=(8, 4, 8), post_radius=2.0)
    c["skin"] = 1e-3
    m, *_ = gpu_setup(c)
    compare_lists(m.lists(), oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"]))


@pytest.mark.parametrize("name", ["c2", "c4", "c3", "c5"])
def test_lists_sampled_full_size(name):
    """Rows of the full-size lists: cell 0, the last cell, cells on each
    periodic face (referred cells) and random cells."""
    c = synth.make(name, 0)
    m, *_ = gpu_setup(c)
    g = m.lists()
    C = c["mesh"]["n_cells"]
    rng = np.random.default_rng(1)
    geo = oracle.cell_geometry(c["mesh"])
    L, per = c["box"]["L"], c["box"]["periodic"]
    face = []
    for d in range(3):
        if per[d]:
            lo_side = np.flatnonzero(geo["lo"][:, d] <= 1e-9)
            hi_side = np.flatnonzero(geo["hi"][:, d] >= L[d] - 1e-9)
            face += [rng.choice(lo_side), rng.choice(hi_side)]
    cells = np.unique(np.r_[0, C - 1, face, rng.choice(C, 10, replace=False)])
    o = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], queries=cells, geo=geo)
    assert g["ties"] == 0 and o["ties"] == 0
    compare_lists(g, o, cells)


def test_lists_full_c3():
    """Every row of the nanochannel's lists (91 680 hexahedra, open y axis,
    removed post columns, periodic x and z) against the oracle."""
    c = synth.make("c3", 0)
    m, *_ = gpu_setup(c)
    g = m.lists()
    o = oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], c["skin"])
    assert g["ties"] == 0 and o["ties"] == 0
    compare_lists(g, o)


def test_lists_slab_c5():
    """Every row of a slab of c5's lists: the 5 % of its 3 072 000 tetrahedra
    whose centres lie nearest the periodic face x = 0 (their referred cells
    included), against the oracle."""
    c = synth.make("c5", 0)
    m, *_ = gpu_setup(c)
    g = m.lists()
    geo = oracle.cell_geometry(c["mesh"])
    x = geo["ctr"].reshape(-1, 3)[:, 0]
    cells = np.flatnonzero(x < np.quantile(x, 0.05))
    o = oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], c["skin"], queries=cells, geo=geo)
    assert g["ties"] == 0 and o["ties"] == 0
    assert len(o["ref_src"]) > 0
    compare_lists(g, o, cells)


def test_uniform_cubes_give_n_c(golden):
    n, w = 6, 2.28
    L = n * w
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    mesh = synth.hex_mesh((n, n, n), (0, 0, 0), (L, L, L), 0.0, np.random.default_rng(0))
    cfg = dict(mesh=mesh, box=box, rc=1.0965 * w, skin=0.0, pos=np.full((1, 3), 1.0),
               species=np.zeros(1, np.int32))
    m, *_ = gpu_setup(cfg)
    g = m.lists()
    pairs = len(g["dil_ids"]) + len(g["ref_ids"]) / 2
    assert pairs == n ** 3 * (golden["N_c"]["1.0965"] - 1) / 2


def test_lists_are_deterministic():
    c = synth.make("t0", 3)
    m, *_ = gpu_setup(c)
    a = m.lists()
    m.build_lists(c["rc"], c["skin"])
    b = m.lists()
    for k in ("dil_off", "dil_ids", "ref_src", "ref_n", "ref_off", "ref_ids"):
        np.testing.assert_array_equal(a[k], b[k])
