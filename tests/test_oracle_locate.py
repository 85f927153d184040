"""Pins for the oracle's point location (CPU only).

On an undistorted grid of cubes the containing hexahedron is the floor of
the coordinates; inside a cube split along its main diagonal, the Kuhn
tetrahedron is fixed by the descending order of the local coordinates.  Ties
(points on faces, edges and vertices) follow the perturbation p + (e, e^2, e^3),
so the floor rule and an x-before-y-before-z order on equal coordinates still
hold exactly; those cases also exercise the exact rational slow path.
"""
import itertools

import numpy as np

import oracle
from paper_cs_0702131_gb300 import synth

N, W = 4, 0.5                 # dyadic spacing: grid planes are exact doubles
BOX = dict(L=np.array([N * W] * 3), periodic=np.array([1, 1, 1], np.int32))
PERMS = list(itertools.permutations((0, 1, 2)))   # axis order of synth's Kuhn tets


def _hex_id(ix, iy, iz):
    return (ix * N + iy) * N + iz


def _expected_hex(p):
    g = np.floor(np.asarray(p) / W).astype(int)
    return _hex_id(*g)


def _expected_tet(p):
    g = np.floor(np.asarray(p) / W).astype(int)
    u = np.asarray(p) / W - g
    perm = tuple(sorted(range(3), key=lambda a: (-u[a], a)))   # ties: x before y before z
    return _hex_id(*g) * 6 + PERMS.index(perm)


def test_hex_grid_generic_points():
    mesh = synth.hex_mesh((N, N, N), (0, 0, 0), BOX["L"], 0.0, np.random.default_rng(0))
    geo = oracle.cell_geometry(mesh)
    p = np.random.default_rng(1).uniform(0, N * W, size=(2000, 3))
    cell, _ = oracle.locate(geo, BOX, p)
    np.testing.assert_array_equal(cell, [_expected_hex(q) for q in p])


def test_hex_grid_ties_and_wrap():
    mesh = synth.hex_mesh((N, N, N), (0, 0, 0), BOX["L"], 0.0, np.random.default_rng(0))
    geo = oracle.cell_geometry(mesh)
    rng = np.random.default_rng(2)
    p = rng.integers(0, 2 * N, size=(400, 3)) * (W / 2)      # on faces, edges, vertices
    cell, wrapped = oracle.locate(geo, BOX, p)
    np.testing.assert_array_equal(cell, [_expected_hex(q) for q in wrapped])
    q = np.array([[N * W, 0.25, 0.25], [-0.25, 0.25, 0.25], [0.25, 2 * N * W + 0.25, 0.25]])
    cell, wrapped = oracle.locate(geo, BOX, q)
    np.testing.assert_array_equal(wrapped, [[0, 0.25, 0.25], [N * W - 0.25, 0.25, 0.25], [0.25, 0.25, 0.25]])
    np.testing.assert_array_equal(cell, [_expected_hex(x) for x in wrapped])


def test_kuhn_tets_generic_and_ties():
    mesh = synth.hex_mesh((N, N, N), (0, 0, 0), BOX["L"], 0.0, np.random.default_rng(0), tets=True)
    geo = oracle.cell_geometry(mesh)
    rng = np.random.default_rng(3)
    p = rng.uniform(0, N * W, size=(1500, 3))
    cell, _ = oracle.locate(geo, BOX, p)
    np.testing.assert_array_equal(cell, [_expected_tet(q) for q in p])
    # on the diagonal faces x = y, y = z, x = z and on grid planes
    t = rng.integers(0, 8 * N, size=(300, 3)) * (W / 8)
    t[:100, 1] = t[:100, 0]
    t[100:200, 2] = t[100:200, 1]
    t[200:, 2] = t[200:, 0]
    cell, _ = oracle.locate(geo, BOX, t)
    np.testing.assert_array_equal(cell, [_expected_tet(q) for q in t])


def test_outside_open_axis():
    box = dict(L=np.array([N * W] * 3), periodic=np.array([1, 0, 1], np.int32))
    mesh = synth.hex_mesh((N, N, N), (0, 0, 0), box["L"], 0.0, np.random.default_rng(0))
    geo = oracle.cell_geometry(mesh)
    p = np.array([[0.3, -0.01, 0.3], [0.3, N * W, 0.3], [0.3, N * W + 1, 0.3], [0.3, 0.0, 0.3]])
    cell, _ = oracle.locate(geo, box, p)
    # y = L_y is the top boundary: the perturbed point lies above it
    np.testing.assert_array_equal(cell, [-1, -1, -1, _expected_hex(p[3])])


def test_jittered_meshes_cover_every_molecule():
    for name in ("c1", "t0", "h0"):
        c = synth.make(name, seed=9)
        geo = oracle.cell_geometry(c["mesh"])
        cell, _ = oracle.locate(geo, c["box"], c["pos"])
        assert np.all(cell >= 0)
        # the centroid of each cell lies in that cell (cells are star-shaped about it)
        cc, _ = oracle.locate(geo, c["box"], geo["ctr"])
        np.testing.assert_array_equal(cc, np.arange(geo["n_cells"]))


def test_bin_order_is_stable_counting_sort():
    cell = np.array([2, 0, 2, 1, 0, 2], np.int32)
    order, off = oracle.bin_order(cell, 4)
    np.testing.assert_array_equal(order, [1, 4, 3, 0, 2, 5])
    np.testing.assert_array_equal(off, [0, 2, 3, 6, 6])
