"""Pins for the autograd-of-oracle adjoint reference (CPU only): its forces
equal the C oracle's, and its vector-Jacobian product equals central finite
differences of sum(v . F) computed with the C oracle."""
import numpy as np

import oracle
from oracle import torch_ref
from paper_cs_0702131_gb300 import synth


def _system(seed=0):
    rng = np.random.default_rng(seed)
    a = synth.A_FCC_08
    L = 4 * a
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    pos = synth.wrap(synth.jitter(synth.fcc_sites(4, 4, 4, a), 0.05, rng), box["L"], box["periodic"])
    sp = np.zeros(len(pos), np.int32)
    sp[rng.permutation(len(pos))[: len(pos) // 2]] = 1
    return pos, sp, np.array([1.0, 1.5]), np.array([1.0, 0.88]), 2.5, box


def test_torch_forces_equal_c_oracle():
    pos, sp, eps, sig, rc, box = _system(1)
    v = np.zeros_like(pos)
    _, _, _, F = torch_ref.vjp(pos, sp, eps, sig, rc, box, v)
    ref = oracle.lj(pos, sp, eps, sig, rc, box)
    assert np.abs(F - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()


def test_vjp_matches_finite_differences():
    pos, sp, eps, sig, rc, box = _system(2)
    rng = np.random.default_rng(5)
    v = rng.normal(size=pos.shape)
    gx, ge, gs, _ = torch_ref.vjp(pos, sp, eps, sig, rc, box, v)
    h = 1e-6

    def phi(p=pos, e=eps, s=sig):
        return float((oracle.lj(p, sp, e, s, rc, box)["F"] * v).sum())

    for k in rng.choice(len(pos), 5, replace=False):
        d = pos - pos[k]
        d -= box["L"] * np.round(d / box["L"])
        if np.any(np.abs(np.linalg.norm(d, axis=1) - rc) < 1e-3):
            continue
        for ax in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, ax] += h
            pm[k, ax] -= h
            fd = (phi(p=pp) - phi(p=pm)) / (2 * h)
            assert abs(fd - gx[k, ax]) <= 1e-5 * max(1.0, abs(gx[k, ax]))
    for s in range(2):
        de = np.zeros(2)
        de[s] = h
        fd = (phi(e=eps + de) - phi(e=eps - de)) / (2 * h)
        assert abs(fd - ge[s]) <= 1e-6 * max(1.0, abs(ge[s]))
        fd = (phi(s=sig + de) - phi(s=sig - de)) / (2 * h)
        assert abs(fd - gs[s]) <= 1e-6 * max(1.0, abs(gs[s]))
