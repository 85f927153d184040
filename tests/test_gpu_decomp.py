"""Processor referral on the CUDA path (§2.1, App. A.2, and the criterion of
§3 that a decomposed run reproduces the serial one).

Each portion of a spatial decomposition runs the library's kernels on its
own molecules plus the halo it receives (the molecules of the remote
source cells of its processor-referred cells, from decomp.halo_plan): a
pair of two owned molecules with Newton's third law, an owned-halo pair
one-sidedly with half its energy and virial.  The halo exchange is done in
one process (each portion's halo is cut from the other portions' molecules,
as the owners would send it); every portion is evaluated through the C ABI
on the GPU, and the portions' owned forces and summed energy and virial
must equal the serial oracle: 1e-12 (FP64) and the FP32 tolerance
(1e-5 of max(|F_ic|, ||F_i||) per component; 1e-6 energy and virial)."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0702131_gb300 import decomp, synth
from paper_cs_0702131_gb300.aica import AicaError, Mesh
from gpu_helpers import assert_forces

pytestmark = pytest.mark.gpu
TOL = {"fp64": (1e-12, 1e-12), "fp32": (1e-5, 1e-6)}


def _portions(name, seed, P, prec):
    c = synth.make(name, seed)
    geo = oracle.cell_geometry(c["mesh"])
    cell, _ = oracle.locate(geo, c["box"], c["pos"])
    m = Mesh(c["mesh"], c["box"])
    m.build_lists(c["rc"], c["skin"])
    lists = m.lists()
    part = decomp.partition(geo["ctr"], P)
    n = len(c["pos"])
    F = np.full((n, 3), np.nan)
    ev = np.zeros(7)
    halo_total = 0
    for r in range(P):
        plan = decomp.halo_plan(lists, part, r)
        own = np.flatnonzero(part[cell] == r)
        halo = decomp.halo_molecules(plan, cell)
        assert np.all(part[cell[halo]] != r)
        halo_total += len(halo)
        idx = np.concatenate([own, halo])
        pos = torch.tensor(c["pos"][idx], dtype=torch.float64, device="cuda")
        sp = torch.tensor(c["species"][idx], dtype=torch.int32, device="cuda")
        m.set_option("n_owned", len(own))
        m.bin(pos, sp)
        Fr, evr, _ = m.forces(c["eps"], c["sigma"], prec)
        F[own] = Fr.double().cpu().numpy()[:len(own)]
        ev += evr.cpu().numpy()
    m.set_option("n_owned", -1)
    return c, m, F, ev, halo_total


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,seed,P", [("t0", 3, 2), ("t0", 3, 3), ("c1", 1, 3), ("h0", 2, 2)])
def test_portions_reproduce_serial(name, seed, P, prec):
    c, m, F, ev, halo = _portions(name, seed, P, prec)
    ref = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    assert halo > 0 and not np.isnan(F).any()
    tf, te = TOL[prec]
    assert_forces(F, ref, tf)
    assert abs(ev[0] - ref["U"]) <= te * ref["Uabs"]
    assert np.all(np.abs(ev[1:] - ref["W"]) <= te * ref["Wabs"])
    m.close()


def test_portion_mode_refuses_paths_without_it():
    c = synth.make("t0", 3)
    m = Mesh(c["mesh"], c["box"])
    m.build_lists(c["rc"], c["skin"])
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    m.set_option("n_owned", len(c["pos"]) // 2)
    m.bin(pos, sp)
    m.set_option("fp32_kernel", 1)
    with pytest.raises(AicaError):
        m.forces(c["eps"], c["sigma"], "fp32")
    m.set_option("fp32_kernel", 0)
    with pytest.raises(AicaError):
        m.forces_backward(c["eps"], c["sigma"], torch.zeros_like(pos), "fp64")
    m.set_option("n_owned", -1)
    m.close()
