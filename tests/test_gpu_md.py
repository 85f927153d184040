"""Velocity-Verlet steps around the GPU hot path (aica_verlet_step) against
the oracle's integrator, and the verification criteria of §3: momentum
conservation and results independent of the mesh."""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import Mesh, aica_kinetic

pytestmark = pytest.mark.gpu
MASS = [1.0]


def _run(c, mesh, v0, dt, steps, prec="fp64", shift=False):
    m = Mesh(mesh, c["box"])
    m.build_lists(c["rc"], c["skin"])
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    vel = torch.tensor(v0, dtype=torch.float64, device="cuda")
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    m.bin(pos, sp, outputs=False)
    F, ev, _ = m.forces(c["eps"], c["sigma"], prec, shift=shift)
    kin = torch.empty(4, dtype=torch.float64, device="cuda")
    aica_kinetic(MASS, sp, vel, kin)
    KE, PE, P = [kin[0].item()], [ev[0].item()], [kin[1:].cpu().numpy()]
    for _ in range(steps):
        m.verlet_step(c["eps"], c["sigma"], MASS, dt, pos, vel, sp, F, prec=prec, ev=ev, kin=kin, shift=shift)
        KE.append(kin[0].item())
        PE.append(ev[0].item())
        P.append(kin[1:].cpu().numpy())
    out = dict(pos=pos.cpu().numpy(), vel=vel.cpu().numpy(), KE=np.array(KE), PE=np.array(PE), P=np.array(P))
    m.close()
    return out


def _start(seed=1):
    c = synth.make("t0", seed)
    v0 = np.random.default_rng(seed + 10).normal(scale=0.7, size=c["pos"].shape)
    return c, v0 - v0.mean(0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_verlet_matches_oracle(prec, tol):
    c, v0 = _start()
    g = _run(c, c["mesh"], v0, 0.002, 20, prec)
    o = oracle.verlet(c["pos"], v0, c["species"], c["eps"], c["sigma"], MASS, c["rc"], c["box"], 0.002, 20)
    assert np.abs(g["pos"] - o["pos"]).max() <= tol
    assert np.abs(g["vel"] - o["vel"]).max() <= tol * 10
    np.testing.assert_allclose(g["KE"], o["KE"], rtol=tol)
    np.testing.assert_allclose(g["PE"], o["PE"], rtol=tol)


def test_results_do_not_depend_on_the_mesh():
    """§3, third criterion: the same molecules on Kuhn tetrahedra and on
    jittered hexahedra follow the same trajectory (FP64)."""
    c, v0 = _start(2)
    L = c["box"]["L"]
    hexes = synth.hex_mesh((5, 5, 5), (0, 0, 0), L, 0.15, np.random.default_rng(9))
    a = _run(c, c["mesh"], v0, 0.002, 100)
    b = _run(c, hexes, v0, 0.002, 100)
    np.testing.assert_allclose(a["KE"], b["KE"], rtol=1e-10)
    np.testing.assert_allclose(a["PE"], b["PE"], rtol=1e-10)
    assert np.abs(a["pos"] - b["pos"]).max() <= 1e-9


def test_momentum_and_energy_are_conserved():
    """Momentum to rounding; total energy with the shifted potential (plain
    truncation makes U jump by u(rc) whenever a pair crosses rc) to the
    second-order error of the scheme."""
    c, v0 = _start(3)
    g = _run(c, c["mesh"], v0, 0.002, 200, shift=True)
    assert np.abs(g["P"] - g["P"][0]).max() <= 1e-12 * np.abs(v0).sum()
    E = g["KE"] + g["PE"]
    assert np.abs(E - E[0]).max() <= 1e-3 * abs(E[0])
