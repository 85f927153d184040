"""Pins for the referring transforms of §2.2.2 and the oracle's sum over
images (CPU only): the tensor of the coupled faces, composition, the
closure's order independence, the box as a special case, and a rotationally
periodic wedge against the explicit full annulus."""
import numpy as np

import oracle
from oracle import transforms as T
from paper_cs_0702131_gb300 import synth


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def test_face_tensor_turns_minus_n_alpha_into_n_beta():
    rng = np.random.default_rng(0)
    for _ in range(50):
        na, nb = _unit(rng.normal(size=3)), _unit(rng.normal(size=3))
        R = T.rotation(na, nb)
        np.testing.assert_allclose(R @ (-na), nb, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
    np.testing.assert_array_equal(T.rotation([1, 0, 0], [-1, 0, 0]), np.eye(3))   # plain periodic box


def test_coupling_maps_face_centre_and_composition():
    na, ca = _unit([0.3, -1.0, 0.2]), np.array([1.0, 2.0, 3.0])
    nb, cb = _unit([-1.0, 0.1, 0.4]), np.array([-4.0, 0.5, 2.0])
    Tab = T.coupling(na, ca, nb, cb)
    np.testing.assert_allclose(T.apply(Tab, ca), cb, atol=1e-12)
    rng = np.random.default_rng(1)
    P = rng.normal(size=(5, 3))
    T2 = (T.rotation(_unit([0, 0, 1.0]), _unit([1.0, 1.0, 0])), np.array([0.5, -1.0, 2.0]))
    np.testing.assert_allclose(T.apply(T.compose(T2, Tab), P), T.apply(T2, T.apply(Tab, P)), atol=1e-12)
    np.testing.assert_allclose(T.apply(T.compose(T.inverse(Tab), Tab), P), P, atol=1e-12)


def test_closure_is_order_independent():
    c = synth.wedge(0)
    g = c["transforms"]
    a = T.closure(g, 4)
    b = T.closure(g[::-1], 4)
    assert len(a) == len(b)
    for t in a:
        assert any(T.same(t, u) for u in b)


def test_box_translations_equal_minimum_image_sum():
    c = synth.make("t0", 3)
    L = c["box"]["L"]
    gens = [(np.eye(3), np.eye(3)[d] * L[d]) for d in range(3)]
    ref = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    img = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], T.closure(gens, 3))
    assert np.abs(img["F"] - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()
    np.testing.assert_allclose(img["U"], ref["U"], rtol=1e-12)
    np.testing.assert_allclose(img["W"], ref["W"], rtol=1e-11, atol=1e-9)
    assert img["row_pairs"] == ref["row_pairs"]


def test_wedge_images_equal_full_annulus():
    """The quarter sector with its two periodic transforms gives each of its
    molecules the forces it has in the explicit annulus of four sectors."""
    c = synth.wedge(1)
    n = len(c["pos"])
    img = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], T.closure(c["transforms"], 6))
    rot = c["transforms"][0]
    full = [c["pos"]]
    for _ in range(3):
        full.append(T.apply(rot, full[-1]))
    full = np.concatenate(full)
    box = dict(L=np.array([100.0, 100.0, c["H"]]), periodic=np.array([0, 0, 1], np.int32))
    ref = oracle.lj(full, np.zeros(len(full), np.int32), c["eps"], c["sigma"], c["rc"], box, idx=np.arange(n))
    assert np.abs(img["F"] - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()
    assert img["row_pairs"] == ref["row_pairs"]
    # deeper compositions add no image within rc
    img8 = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], T.closure(c["transforms"], 8))
    np.testing.assert_array_equal(img8["F"], img["F"])


def test_image_rows_equal_full():
    c = synth.wedge(3)
    xf = T.closure(c["transforms"], 6)
    full = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], xf)
    idx = np.array([0, 5, 17, len(c["pos"]) - 1])
    part = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], xf, idx=idx)
    np.testing.assert_array_equal(part["F"], full["F"][idx])
