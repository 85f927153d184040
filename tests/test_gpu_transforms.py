"""General referring transforms (§2.2.2) on the GPU: a rotationally periodic
wedge against the oracle's sum over images."""
import numpy as np
import pytest
import torch

import oracle
from oracle import transforms as T
from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import AicaError, Mesh, aica_coupling_transform

pytestmark = pytest.mark.gpu


def test_coupling_transform_matches_the_oracle():
    na, ca = np.array([0.0, -1.0, 0.0]), np.array([8.0, 0.0, 4.0])
    nb, cb = np.array([-1.0, 0.0, 0.0]), np.array([0.0, 8.0, 4.0])
    R, y = aica_coupling_transform(na, ca, nb, cb)
    Ro, yo = T.coupling(na, ca, nb, cb)
    np.testing.assert_allclose(R, Ro, atol=1e-15)
    np.testing.assert_allclose(y, yo, atol=1e-12)
    rng = np.random.default_rng(2)
    for _ in range(20):
        a, b = rng.normal(size=3), rng.normal(size=3)
        R, _ = aica_coupling_transform(a, np.zeros(3), b, np.zeros(3))
        np.testing.assert_allclose(R, T.rotation(a, b), atol=1e-13)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("seed", [1, 2])
def test_wedge_forces_equal_oracle(seed, prec, tol):
    c = synth.wedge(seed)
    m = Mesh(c["mesh"], c["box"])
    m.set_transforms(c["transforms"])
    m.build_lists(c["rc"], c["skin"])
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    m.bin(pos, sp)
    ref = oracle.lj_images(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], T.closure(c["transforms"], 6))
    F, ev, cnt = m.forces(c["eps"], c["sigma"], prec)
    err = np.abs(F.double().cpu().numpy() - ref["F"]) / ref["Fabs"][:, None]
    assert err.max() <= tol
    assert abs(ev[0].item() - ref["U"]) <= (1e-12 if prec == "fp64" else 1e-6) * ref["Uabs"]
    assert np.all(np.abs(ev[1:].cpu().numpy() - ref["W"]) <= (1e-12 if prec == "fp64" else 1e-6) * ref["Wabs"])
    k = cnt.cpu().numpy()
    assert 2 * (k[3] + k[4]) + k[5] == ref["row_pairs"]
    lists = m.lists()
    assert lists["ties"] == 0 and len(lists["ref_src"]) > 0
    m.close()


def test_transforms_need_a_box_without_periodic_axes():
    c = synth.make("t0", 0)
    m = Mesh(c["mesh"], c["box"])
    with pytest.raises(AicaError):
        m.set_transforms([(np.eye(3), np.array([1.0, 0, 0]))])
    m.close()
