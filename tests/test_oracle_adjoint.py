"""Pins for the autograd-of-oracle adjoint reference (CPU only): its forces
equal the C oracle's, and its vector-Jacobian product equals central finite
differences of sum(v . F) computed with the C oracle."""
import numpy as np

import oracle
from oracle import torch_ref
from oracle import transforms as T
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


def _wedge(seed, species_count=2):
    c = synth.wedge(seed)
    rng = np.random.default_rng(seed + 10)
    sp = rng.integers(0, species_count, len(c["pos"])).astype(np.int32)
    eps = np.linspace(1.0, 1.5, species_count)
    sig = np.linspace(1.0, 0.88, species_count)
    return c, sp, eps, sig


def test_image_forces_equal_c_oracle():
    c, sp, eps, sig = _wedge(1)
    tr = T.closure(c["transforms"], 6)
    _, _, _, F = torch_ref.image_vjp(c["pos"], sp, eps, sig, c["rc"], tr, np.zeros_like(c["pos"]))
    ref = oracle.lj_images(c["pos"], sp, eps, sig, c["rc"], tr)
    assert np.abs(F - ref["F"]).max() <= 1e-12 * ref["Fabs"].max()


def test_image_vjp_matches_finite_differences():
    """Central differences of sum(v . F) from the C oracle's image sum: the
    source molecule of a rotated image gets its gradient through R^T."""
    c, sp, eps, sig = _wedge(2)
    tr = T.closure(c["transforms"], 6)
    pos, rc = c["pos"], c["rc"]
    rng = np.random.default_rng(7)
    v = rng.normal(size=pos.shape)
    gx, ge, gs, _ = torch_ref.image_vjp(pos, sp, eps, sig, rc, tr, v)
    h = 1e-6

    def phi(p=pos, e=eps, s=sig):
        return float((oracle.lj_images(p, sp, e, s, rc, tr)["F"] * v).sum())

    # molecules near the wedge's cut faces, whose images carry rotations
    ang = np.arctan2(pos[:, 1], pos[:, 0])
    near = np.nonzero((ang < 0.3) | (ang > np.pi / 2 - 0.3))[0]
    checked = 0
    for k in rng.choice(near, 6, replace=False):
        q = np.concatenate([pos @ np.asarray(R).T + np.asarray(y) for R, y in tr])
        if np.any(np.abs(np.linalg.norm(q - pos[k], axis=1) - rc) < 1e-3):
            continue
        checked += 1
        for ax in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, ax] += h
            pm[k, ax] -= h
            fd = (phi(p=pp) - phi(p=pm)) / (2 * h)
            assert abs(fd - gx[k, ax]) <= 1e-5 * max(1.0, abs(gx[k, ax]))
    assert checked >= 3
    for s in range(2):
        de = np.zeros(2)
        de[s] = h
        fd = (phi(e=eps + de) - phi(e=eps - de)) / (2 * h)
        assert abs(fd - ge[s]) <= 1e-6 * max(1.0, abs(ge[s]))
        fd = (phi(s=sig + de) - phi(s=sig - de)) / (2 * h)
        assert abs(fd - gs[s]) <= 1e-6 * max(1.0, abs(gs[s]))


def test_vjp_rows_equal_full_vjp():
    pos, sp, eps, sig, rc, box = _system(3)
    v = np.random.default_rng(8).normal(size=pos.shape)
    gx, _, _, _ = torch_ref.vjp(pos, sp, eps, sig, rc, box, v)
    idx = np.array([0, 5, 17, len(pos) - 1])
    rows = torch_ref.vjp_rows(pos, sp, eps, sig, rc, box, v, idx)
    assert np.abs(rows - gx[idx]).max() <= 1e-12 * np.abs(gx).max()
