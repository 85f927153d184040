"""The seeded generators: sizes, validity of the meshes, determinism."""
import numpy as np

from paper_cs_0702131_gb300 import synth


def _cell_volumes(mesh):
    P = mesh["points"]
    fo, fv = mesh["face_offsets"], mesh["face_vertices"]
    vol = np.zeros(mesh["n_cells"])
    for f in range(len(mesh["owner"])):
        vs = fv[fo[f]:fo[f + 1]]
        for i in range(1, len(vs) - 1):
            t = np.dot(P[vs[0]], np.cross(P[vs[i]], P[vs[i + 1]])) / 6.0   # divergence theorem
            vol[mesh["owner"][f]] += t
            if mesh["neighbour"][f] >= 0:
                vol[mesh["neighbour"][f]] -= t
    return vol


def test_sizes_and_boxes():
    c = synth.make("c1")
    assert c["pos"].shape == (2048, 3) and c["mesh"]["n_cells"] == 216
    np.testing.assert_allclose(c["box"]["L"], 8 * synth.A_FCC_08)
    c = synth.make("t0")
    assert c["pos"].shape == (864, 3) and c["mesh"]["n_cells"] == 384
    c = synth.make("c4")
    assert c["pos"].shape == (65536, 3) and np.bincount(c["species"]).tolist() == [32768, 32768]


def test_meshes_are_closed_and_fill_the_box():
    for name in ("c1", "t0", "h0"):
        c = synth.make(name, seed=3)
        m = c["mesh"]
        vol = _cell_volumes(m)
        assert np.all(vol > 0)
        np.testing.assert_allclose(vol.sum(), np.prod(c["box"]["L"]), rtol=1e-12)
        inside = (c["pos"] >= 0) & (c["pos"] < c["box"]["L"])
        assert inside.all()


def test_deterministic():
    a, b = synth.make("t0", seed=5), synth.make("t0", seed=5)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["mesh"]["points"], b["mesh"]["points"])
    assert not np.array_equal(a["pos"], synth.make("t0", seed=6)["pos"])


def test_nanochannel_small():
    c = synth.nanochannel(0, nfcc=(12, 4, 12), hex_shape=(8, 4, 8), post_radius=2.0)
    assert c["box"]["periodic"].tolist() == [1, 0, 1]
    assert c["wall"].sum() > 0 and (~c["wall"]).sum() > 0
    vol = _cell_volumes(c["mesh"])
    assert np.all(vol > 0)
