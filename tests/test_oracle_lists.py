"""Pins for the oracle's cell lists (CPU only).

Known distances between simple polyhedra, the k = 5 loop order of App. A.1,
N_c on uniform cubic meshes (§2.4), completeness (the AICA loops over the
lists reproduce the all-pairs sum), referred-cell symmetry, and agreement of
the sampled and the full computation.
"""
import numpy as np
import pytest

import oracle
from paper_cs_0702131_gb300 import synth

OPEN = dict(L=np.array([100.0, 100.0, 100.0]), periodic=np.array([0, 0, 0], np.int32))


def _d2_two_cells(points, cells):
    mesh = synth.cells_to_mesh(points, cells)
    geo = oracle.cell_geometry(mesh)
    A, B, N, d2, _ = oracle.cell_pairs(geo, OPEN, 50.0, queries=[0], use_bound=False)
    assert list(B) == [1]
    return d2[0]


@pytest.mark.parametrize("off,expect", [
    ((1.3, 0, 0), 0.09),                       # face-face gap 0.3
    ((1.3, 1.4, 0), 0.09 + 0.16),             # parallel edges
    ((1.3, 1.4, 1.2), 0.09 + 0.16 + 0.04),    # corner-corner
    ((1.0, 0, 0), 0.0),                        # shared face
    ((1.0, 1.0, 1.0), 0.0),                    # shared corner
])
def test_cube_cube_distance(off, expect):
    pts, cells = synth.cube_cells([(0, 0, 0), off])
    np.testing.assert_allclose(_d2_two_cells(pts, cells), expect, rtol=1e-12, atol=1e-15)


def test_vertex_to_face_interior_distance():
    h = 0.37
    pts, cells = synth.cube_cells([(0, 0, 0)])
    tet = np.array([[0.5, 0.5, 1 + h], [0, 0, 3], [1, 0, 3], [0.5, 1, 3]])
    P = np.vstack([pts, tet])
    cells = [list(range(8)), [8, 9, 10, 11]]
    mesh = synth.cells_to_mesh(P, [cells[0]])             # cube alone as a hex mesh
    tmesh = synth.cells_to_mesh(P, [cells[1]])
    # join the two single-cell meshes
    m = dict(points=P, n_cells=2)
    m["face_offsets"] = np.r_[mesh["face_offsets"], tmesh["face_offsets"][1:] + mesh["face_offsets"][-1]]
    m["face_vertices"] = np.r_[mesh["face_vertices"], tmesh["face_vertices"]]
    m["owner"] = np.r_[mesh["owner"], tmesh["owner"] + 1]
    m["neighbour"] = np.r_[mesh["neighbour"], tmesh["neighbour"]]
    geo = oracle.cell_geometry(m)
    _, B, _, d2, _ = oracle.cell_pairs(geo, OPEN, 50.0, queries=[0], use_bound=False)
    np.testing.assert_allclose(d2[0], h * h, rtol=1e-12)
    # edge above the top face, crossing it at height h: edge-edge distance
    tet2 = np.array([[-1, 0.5, 1 + h], [2, 0.5, 1 + h], [0.5, 0.5, 4], [0.5, 1.5, 3]])
    P2 = np.vstack([pts, tet2])
    t2 = synth.cells_to_mesh(P2, [[8, 9, 10, 11]])
    m2 = dict(m, points=P2, face_vertices=np.r_[mesh["face_vertices"], t2["face_vertices"]],
              face_offsets=np.r_[mesh["face_offsets"], t2["face_offsets"][1:] + mesh["face_offsets"][-1]])
    geo2 = oracle.cell_geometry(m2)
    _, B, _, d2, _ = oracle.cell_pairs(geo2, OPEN, 50.0, queries=[0], use_bound=False)
    np.testing.assert_allclose(d2[0], h * h, rtol=1e-12)


def test_dil_loop_order_k5(golden):
    """App. A.1 table: five mutually interacting cells give DIL(i) = i+1..4."""
    pts, cells = synth.cube_cells([(0.3 * i, 0, 0) for i in range(5)], size=0.2)
    mesh = synth.cells_to_mesh(pts, cells)
    L = oracle.cell_lists(mesh, OPEN, rc=2.5, skin=0.0)
    for i in range(5):
        got = list(L["dil_ids"][L["dil_off"][i]:L["dil_off"][i + 1]])
        assert got == golden["dil_k5"][str(i)]
    assert len(L["ref_src"]) == 0


@pytest.mark.parametrize("x", ["0.877", "1.0965", "1.5"])
def test_nc_uniform_cubic_mesh(golden, x):
    """§2.4: in a uniform mesh of cubes of side w a cell interacts with N_c(rc/w) - 1 others."""
    n, w = 6, 2.28
    L = n * w
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    mesh = synth.hex_mesh((n, n, n), (0, 0, 0), (L, L, L), 0.0, np.random.default_rng(0))
    rc = float(x) * w
    geo = oracle.cell_geometry(mesh)
    A, B, N, d2, ties = oracle.cell_pairs(geo, box, rc, use_bound=True)
    assert ties == 0
    per_cell = np.bincount(A, minlength=n ** 3)
    assert np.all(per_cell == golden["N_c"][x] - 1)
    lists = oracle.cell_lists(mesh, box, rc, 0.0, geo=geo)
    unique_pairs = len(lists["dil_ids"]) + len(lists["ref_ids"]) / 2
    assert unique_pairs == n ** 3 * (golden["N_c"][x] - 1) / 2


def test_bound_does_not_change_lists():
    c = synth.make("t0")
    geo = oracle.cell_geometry(c["mesh"])
    a = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo, use_bound=True)
    b = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo, use_bound=False)
    for k in ("dil_off", "dil_ids", "ref_src", "ref_n", "ref_off", "ref_ids"):
        np.testing.assert_array_equal(a[k], b[k])


def _binned(c, geo):
    cell, w = oracle.locate(geo, c["box"], c["pos"])
    assert np.all(cell >= 0)
    order, off = oracle.bin_order(cell, geo["n_cells"])
    return order, off, w[order]


@pytest.mark.parametrize("name", ["t0", "c1", "h0"])
def test_lists_are_complete(name):
    """The §2.3 loops over the lists reproduce the all-pairs sum: no pair is missed
    and none is counted twice (real-referred pairs from both of their sides)."""
    c = synth.make(name, seed=11)
    geo = oracle.cell_geometry(c["mesh"])
    lists = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo)
    order, off, xs = _binned(c, geo)
    a = oracle.aica_loop(lists, off, xs, c["species"][order], c["eps"], c["sigma"], c["rc"], c["box"])
    ref = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    F = np.empty_like(a["F"])
    F[order] = a["F"]
    assert np.abs(F - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()
    np.testing.assert_allclose(a["U"], ref["U"], rtol=1e-12)
    np.testing.assert_allclose(a["W"], ref["W"], rtol=1e-11, atol=1e-9)
    cnt = a["counts"]
    assert cnt[5] % 2 == 0
    assert cnt[3] + cnt[4] + cnt[5] // 2 == ref["pairs"]


def test_list_invariants():
    c = synth.make("c1", seed=4)
    L = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"])
    C = c["mesh"]["n_cells"]
    for i in range(C):
        d = L["dil_ids"][L["dil_off"][i]:L["dil_off"][i + 1]]
        assert np.all(d > i) and np.all(np.diff(d) > 0)       # j > i, ascending, never self
    assert np.all(L["ref_n"].any(axis=1))
    entries = set()
    for M in range(len(L["ref_src"])):
        n = tuple(L["ref_n"][M])
        for J in L["ref_ids"][L["ref_off"][M]:L["ref_off"][M + 1]]:
            entries.add((int(L["ref_src"][M]), n, int(J)))
    mirror = {(J, tuple(-np.array(n)), c_) for (c_, n, J) in entries}
    assert entries == mirror                                  # (c, n) sees J  <=>  (J, -n) sees c
    keys = [(int(s),) + tuple(n) for s, n in zip(L["ref_src"], L["ref_n"])]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_vertex_rule_lists_equal_brute_force_and_are_contained():
    """The oracle's vertex-vertex criterion (§2.2, App. A.1) lists exactly the
    (A, B, n) with a vertex pair closer than rc + skin (numpy brute force),
    and the minimum-distance lists always contain them (d_min <= any vertex
    distance)."""
    c = synth.make("t0", seed=2)
    geo = oracle.cell_geometry(c["mesh"])
    thr = c["rc"] + c["skin"]
    rng = np.random.default_rng(0)
    q = np.sort(rng.choice(geo["n_cells"], 12, replace=False))
    A, B, N, _, _ = oracle.cell_pairs(geo, c["box"], thr, queries=q)
    listed = set(zip(A.tolist(), B.tolist(), map(tuple, N.tolist())))
    Av, Bv, Nv, _, _ = oracle.cell_pairs(geo, c["box"], thr, queries=q, criterion="vertex")
    vertex = set(zip(Av.tolist(), Bv.tolist(), map(tuple, Nv.tolist())))
    V = [geo["vtx"][geo["vtx_off"][i]:geo["vtx_off"][i + 1]] for i in range(geo["n_cells"])]
    L = c["box"]["L"]
    brute = set()
    for A0 in q:
        for B0 in range(geo["n_cells"]):
            for n in np.ndindex(3, 3, 3):
                n = np.array(n) - 1
                if A0 == B0 and not n.any():
                    continue
                d = V[A0][:, None, :] - (V[B0][None, :, :] + n * L)
                if np.sqrt((d * d).sum(-1)).min() < thr:
                    brute.add((int(A0), B0, tuple(int(x) for x in n)))
    assert vertex == brute
    assert vertex <= listed
    assert len(vertex) < len(listed)      # on tetrahedra the vertex rule drops cell pairs


def _twisted_pair(h=1.0):
    """Two tetrahedra whose long edges cross at distance h while every vertex
    pair is farther than 3.8: the slivers of the paper's twisted-mesh figure."""
    pts = np.array([[-3, 0, 0], [3, 0, 0], [0, -0.5, -2], [0, 0.5, -2],
                    [0, -3, h], [0, 3, h], [-0.5, 0, h + 2], [0.5, 0, h + 2]], float) + 10.0
    return synth.cells_to_mesh(pts, np.array([[0, 1, 2, 3], [4, 5, 6, 7]]))


def test_vertex_rule_misses_twisted_cells():
    """§2.2: searching from vertices only can miss interacting slivers; the
    minimum-distance criterion does not.  Two molecules 1.2 apart across the
    crossing edges: the AICA loops over the vertex lists miss their pair."""
    mesh = _twisted_pair()
    lv = oracle.cell_lists(mesh, OPEN, rc=2.5, skin=0.0, criterion="vertex")
    lm = oracle.cell_lists(mesh, OPEN, rc=2.5, skin=0.0)
    assert list(lv["dil_ids"]) == [] and list(lm["dil_ids"]) == [1]
    geo = oracle.cell_geometry(mesh)
    pos = np.array([[10.0, 10.0, 9.9], [10.0, 10.0, 11.1]])    # inside cell 0 and cell 1
    cell, xs = oracle.locate(geo, OPEN, pos)
    assert list(cell) == [0, 1]
    sp = np.zeros(2, np.int32)
    order, off = oracle.bin_order(cell, 2)
    eps, sig = np.array([1.0]), np.array([1.0])
    av = oracle.aica_loop(lv, off, xs[order], sp, eps, sig, 2.5, OPEN)
    am = oracle.aica_loop(lm, off, xs[order], sp, eps, sig, 2.5, OPEN)
    ref = oracle.lj(pos, sp, eps, sig, 2.5, OPEN)
    assert ref["pairs"] == 1 and am["counts"][4] == 1 and av["counts"][4] == 0
    assert np.all(av["F"] == 0.0)
    np.testing.assert_allclose(am["U"], ref["U"], rtol=1e-12)


def test_sampled_queries_equal_full():
    c = synth.make("t0", seed=6)
    geo = oracle.cell_geometry(c["mesh"])
    full = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo)
    q = [3, 100, 383]
    part = oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], queries=q, geo=geo)
    for j, i in enumerate(q):
        np.testing.assert_array_equal(part["dil_ids"][part["dil_off"][j]:part["dil_off"][j + 1]],
                                      full["dil_ids"][full["dil_off"][i]:full["dil_off"][i + 1]])
    sel = np.isin(full["ref_src"], q)
    np.testing.assert_array_equal(part["ref_src"], full["ref_src"][sel])
    np.testing.assert_array_equal(part["ref_n"], full["ref_n"][sel])


def _same_lists(a, b):
    for k in ("cells", "dil_off", "dil_ids", "ref_src", "ref_n", "ref_off", "ref_ids"):
        np.testing.assert_array_equal(np.asarray(a[k]).reshape(-1), np.asarray(b[k]).reshape(-1), err_msg=k)
    assert a["ties"] == b["ties"]


@pytest.mark.parametrize("name,seed", [("t0", 0), ("t0", 5), ("c1", 0), ("h0", 1)])
def test_full_size_search_equals_brute_force(name, seed):
    """cell_lists_full (candidates from a bucket grid of cell centres, for the
    full-size list comparisons) gives exactly the brute-force lists: all
    cells, a subset of query cells, and the paper's vertex criterion."""
    c = synth.make(name, seed)
    geo = oracle.cell_geometry(c["mesh"])
    _same_lists(oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo),
                oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], c["skin"], geo=geo))
    q = np.unique(np.random.default_rng(seed).choice(geo["n_cells"], 40, replace=False))
    _same_lists(oracle.cell_lists(c["mesh"], c["box"], c["rc"], c["skin"], queries=q, geo=geo),
                oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], c["skin"], queries=q, geo=geo))
    _same_lists(oracle.cell_lists(c["mesh"], c["box"], c["rc"], 0.3, geo=geo, criterion="vertex"),
                oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], 0.3, geo=geo, criterion="vertex"))


def test_full_size_search_open_axis_and_removed_cells():
    c = synth.nanochannel(2, nfcc=(12, 4, 12), hex_shape=(8, 4, 8), post_radius=2.0)
    geo = oracle.cell_geometry(c["mesh"])
    _same_lists(oracle.cell_lists(c["mesh"], c["box"], c["rc"], 1e-3, geo=geo),
                oracle.cell_lists_full(c["mesh"], c["box"], c["rc"], 1e-3, geo=geo))
