"""Invariants of the method on the GPU: the same net force whatever the mesh
(§2.3, criterion 3 of §3), periodic replication (the single-device analogue
of the serial = parallel criterion of §3), Newton's third law."""
import numpy as np
import pytest

from paper_cs_0702131_gb300 import synth
from gpu_helpers import gpu_setup

pytestmark = pytest.mark.gpu


def _forces(c, prec="fp64"):
    m, *_ = gpu_setup(c)
    F, ev, cnt = m.forces(c["eps"], c["sigma"], prec)
    cnt = cnt.cpu().numpy()
    return F.double().cpu().numpy(), ev.cpu().numpy(), cnt[3] + cnt[4] + cnt[5]


def test_mesh_independence():
    base = synth.make("c1", 0)
    L = base["box"]["L"]
    meshes = [base["mesh"],
              synth.hex_mesh((6, 6, 6), (0, 0, 0), L, 0.15, np.random.default_rng(9)),
              synth.hex_mesh((4, 4, 4), (0, 0, 0), L, 0.15, np.random.default_rng(3), tets=True),
              synth.hex_mesh((3, 5, 4), (0, 0, 0), L, 0.1, np.random.default_rng(4))]
    # the first mesh again with a random cell numbering
    perm = np.random.default_rng(5).permutation(base["mesh"]["n_cells"])
    inv = np.argsort(perm)
    pm = dict(base["mesh"])
    pm["owner"] = inv[base["mesh"]["owner"]]
    nb = base["mesh"]["neighbour"].copy()
    nb[nb >= 0] = inv[nb[nb >= 0]]
    pm["neighbour"] = nb
    meshes.append(pm)
    F0, ev0, n0 = _forces(dict(base, mesh=meshes[0]))
    scale = np.abs(F0).max()
    for mesh in meshes[1:]:
        F, ev, n = _forces(dict(base, mesh=mesh))
        assert n == n0
        assert np.abs(F - F0).max() <= 1e-12 * scale * 10
        assert abs(ev[0] - ev0[0]) <= 1e-12 * abs(ev0[0]) * 10


def test_periodic_replication():
    c = synth.make("c1", 2)
    L = c["box"]["L"]
    big = dict(c)
    big["pos"] = np.vstack([c["pos"], c["pos"] + [L[0], 0, 0]])
    big["species"] = np.r_[c["species"], c["species"]]
    big["box"] = dict(L=np.array([2 * L[0], L[1], L[2]]), periodic=c["box"]["periodic"])
    big["mesh"] = synth.hex_mesh((12, 6, 6), (0, 0, 0), big["box"]["L"], 0.15, np.random.default_rng(1))
    F1, ev1, n1 = _forces(c)
    F2, ev2, n2 = _forces(big)
    n = len(c["pos"])
    scale = np.abs(F1).max()
    assert np.abs(F2[:n] - F1).max() <= 1e-11 * scale
    assert np.abs(F2[n:] - F1).max() <= 1e-11 * scale
    assert n2 == 2 * n1
    np.testing.assert_allclose(ev2, 2 * ev1, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_newton_third_law(prec, tol):
    c = synth.make("h0", 6)
    F, ev, n = _forces(c, prec)
    assert np.abs(F.sum(0)).max() <= tol * np.abs(F).sum()
