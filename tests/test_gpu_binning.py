"""GPU binning against the oracle: cell ids, binned order and offsets bit-exact."""
import numpy as np
import pytest
import torch

from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import AicaError, Mesh
from gpu_helpers import gpu_setup, oracle_all

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["t0", "c1", "h0", "c4", "c2", "c3", "c5"])
def test_binning_equals_oracle(name):
    """Every molecule's cell, the binned order and the cell offsets, at full
    size (c3: 1.16 M molecules with wall layers on lattice-aligned faces;
    c5: 8.4 M molecules in 3.07 M tetrahedra)."""
    c = synth.make(name, 2)
    m, pos, sp, (cell_of, order, cell_off) = gpu_setup(c)
    o = oracle_all(c, lists=False)
    np.testing.assert_array_equal(cell_of, o["cell"])
    np.testing.assert_array_equal(order, o["order"])
    np.testing.assert_array_equal(cell_off, o["cell_off"])


@pytest.mark.parametrize("name,dist", [("c2", 0.01), ("c2", 0.5), ("c5", 0.5)])
def test_rebinning_after_displacement(name, dist):
    """Re-binning uses the previous cells as a search hint; the result stays exact."""
    c = synth.make(name, 4)
    m, pos, sp, _ = gpu_setup(c)
    rng = np.random.default_rng(7)
    c["pos"] = synth.random_displacement(c["pos"], dist, rng, c["box"]["L"], c["box"]["periodic"])
    cell_of, order, cell_off = m.bin(torch.tensor(c["pos"], device="cuda"), sp)
    o = oracle_all(c, lists=False)
    np.testing.assert_array_equal(cell_of.cpu().numpy(), o["cell"])
    np.testing.assert_array_equal(order.cpu().numpy(), o["order"])
    np.testing.assert_array_equal(cell_off.cpu().numpy(), o["cell_off"])


@pytest.mark.parametrize("tets", [False, True])
def test_ties_on_faces_edges_vertices(tets):
    N, W = 4, 0.5
    box = dict(L=np.array([N * W] * 3), periodic=np.array([1, 1, 1], np.int32))
    mesh = synth.hex_mesh((N, N, N), (0, 0, 0), box["L"], 0.0, np.random.default_rng(0), tets=tets)
    rng = np.random.default_rng(3)
    p = rng.integers(0, 8 * N, size=(3000, 3)) * (W / 8)
    p[:500, 1] = p[:500, 0]
    p[500:1000, 2] = p[500:1000, 1]
    p[1000:1500, 2] = p[1000:1500, 0]
    p[1500:1600] = rng.integers(-8, 8 * N + 8, size=(100, 3)) * (W / 8)   # wrap through the box faces
    cfg = dict(mesh=mesh, box=box, pos=p, species=np.zeros(len(p), np.int32), rc=0.4, skin=0.0)
    m, pos, sp, (cell_of, order, cell_off) = gpu_setup(cfg)
    o = oracle_all(cfg, lists=False)
    np.testing.assert_array_equal(cell_of, o["cell"])
    np.testing.assert_array_equal(order, o["order"])


def test_outside_molecules_reported():
    c = synth.nanochannel(0, nfcc=(12, 4, 12), hex_shape=(8, 4, 8), post_radius=2.0)
    pos = c["pos"].copy()
    pos[5, 1] = 100.0            # far above the open y boundary
    m = Mesh(c["mesh"], c["box"])
    m.build_lists(2.5, 1e-3)
    P = torch.tensor(pos, device="cuda")
    S = torch.zeros(len(pos), dtype=torch.int32, device="cuda")
    with pytest.raises(AicaError) as e:
        m.bin(P, S)
    assert e.value.name == "AICA_ERR_OUTSIDE_MESH"
    m.set_deferred(True)
    cell_of, order, cell_off = m.bin(P, S)
    assert cell_of[5].item() == -1 and cell_off[-1].item() == len(pos) - 1
    with pytest.raises(AicaError):
        m.check()
    F, ev, cnt = m.forces([1.0], [1.0], "fp64")
    assert torch.all(F[5] == 0)
    # deferred errors accumulate over calls until check() reports and clears them
    m.bin(P, S)
    Q = P.clone()
    Q[5] = Q[4]
    m.bin(Q, S)
    with pytest.raises(AicaError) as e:
        m.check()
    assert e.value.name == "AICA_ERR_OUTSIDE_MESH"
    m.bin(Q, S)
    m.check()


def test_repeated_binning_stays_exact():
    """Several binnings in a row of moving molecules: the single-pass scan of
    the cell counts (6 tiles of cells here) runs once per call, and molecules
    that left their cell are found across the face they crossed or by the
    exact search."""
    c = synth._lj_fluid((16, 16, 16), synth.A_FCC_08, (12, 12, 12), True, 2.5, 5)
    c["skin"] = 1e-3
    m, pos, sp, _ = gpu_setup(c)
    rng = np.random.default_rng(9)
    for dist in (0.02, 0.05, 0.3, 0.02):
        c["pos"] = synth.random_displacement(c["pos"], dist, rng, c["box"]["L"], c["box"]["periodic"])
        cell_of, order, cell_off = m.bin(torch.tensor(c["pos"], device="cuda"), sp)
        o = oracle_all(c, lists=False)
        np.testing.assert_array_equal(cell_of.cpu().numpy(), o["cell"])
        np.testing.assert_array_equal(order.cpu().numpy(), o["order"])
        np.testing.assert_array_equal(cell_off.cpu().numpy(), o["cell_off"])
