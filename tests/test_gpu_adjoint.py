"""The hand-written adjoint against the autograd-of-oracle reference, finite
differences and torch.autograd.gradcheck (FP64)."""
import numpy as np
import pytest
import torch

from oracle import torch_ref
from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import LJForce, Mesh
from gpu_helpers import gpu_setup

pytestmark = pytest.mark.gpu


def _two_species_small(seed=0, n=4, hexes=3, rc=2.5):
    rng = np.random.default_rng(seed)
    a = synth.A_FCC_08
    L = n * a
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    pos = synth.wrap(synth.jitter(synth.fcc_sites(n, n, n, a), 0.05, rng), box["L"], box["periodic"])
    sp = np.zeros(len(pos), np.int32)
    sp[rng.permutation(len(pos))[: len(pos) // 2]] = 1
    mesh = synth.hex_mesh((hexes,) * 3, (0, 0, 0), box["L"], 0.15, rng)
    return dict(pos=pos, species=sp, eps=np.array([1.0, 1.5]), sigma=np.array([1.0, 0.88]), rc=rc, box=box,
                mesh=mesh, skin=1e-3)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("which", ["t0", "mix"])
def test_vjp_matches_autograd_of_oracle(which, prec, tol):
    c = synth.make("t0", 2) if which == "t0" else _two_species_small(1)
    m, *_ = gpu_setup(c)
    v = np.random.default_rng(3).normal(size=c["pos"].shape)
    gx, ge, gs, _ = torch_ref.vjp(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], v)
    dt = torch.float64 if prec == "fp64" else torch.float32
    gp, ge_g, gs_g = m.forces_backward(c["eps"], c["sigma"], torch.tensor(v, dtype=dt, device="cuda"), prec)
    assert np.abs(gp.double().cpu().numpy() - gx).max() <= tol * np.abs(gx).max()
    np.testing.assert_allclose(ge_g.cpu().numpy(), ge, rtol=tol, atol=tol * np.abs(ge).max())
    np.testing.assert_allclose(gs_g.cpu().numpy(), gs, rtol=tol, atol=tol * np.abs(gs).max())


def test_force_matching_loss_c4():
    """c4: loss = sum |F - F_t|^2, F_t from parameters scaled by 1.05; backward
    against the autograd reference and FP64 central differences."""
    c = synth.make("c4", 0)
    m, pos, sp, _ = gpu_setup(c)
    F, _, _ = m.forces(c["eps"], c["sigma"], "fp64")
    Ft, _, _ = m.forces(c["eps"] * 1.05, c["sigma"] * 1.05, "fp64")
    v = 2 * (F - Ft)                         # dL/dF
    gp, ge_g, gs_g = m.forces_backward(c["eps"], c["sigma"], v, "fp64")
    gx, ge, gs, _ = torch_ref.vjp(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], v.cpu().numpy())
    assert np.abs(gp.cpu().numpy() - gx).max() <= 1e-10 * np.abs(gx).max()
    np.testing.assert_allclose(ge_g.cpu().numpy(), ge, rtol=1e-10)
    np.testing.assert_allclose(gs_g.cpu().numpy(), gs, rtol=1e-10)

    def loss(eps, sig, p=None):
        if p is not None:
            m.bin(p, sp, outputs=False)
        Fx, _, _ = m.forces(eps, sig, "fp64")
        return float(((Fx - Ft) ** 2).sum())

    h = 1e-6
    for s in range(2):
        d = np.zeros(2)
        d[s] = h
        fd = (loss(c["eps"] + d, c["sigma"]) - loss(c["eps"] - d, c["sigma"])) / (2 * h)
        assert abs(fd - ge_g[s].item()) <= 1e-5 * abs(ge_g[s].item()) + 1e-6
        fd = (loss(c["eps"], c["sigma"] + d) - loss(c["eps"], c["sigma"] - d)) / (2 * h)
        assert abs(fd - gs_g[s].item()) <= 1e-5 * abs(gs_g[s].item()) + 1e-6
    # position checks: the FP64 forces are summed with atomics, so the loss
    # itself differs between repeated evaluations in its last bits; the
    # difference quotient carries that noise divided by h (measured here)
    L0 = loss(c["eps"], c["sigma"])
    noise = max(abs(loss(c["eps"], c["sigma"]) - L0) for _ in range(4))
    hx = 1e-5
    rng = np.random.default_rng(2)
    for k in rng.choice(len(c["pos"]), 64, replace=False):
        ax = int(rng.integers(3))
        p = pos.clone()
        p[k, ax] += hx
        lp = loss(c["eps"], c["sigma"], p)
        p[k, ax] -= 2 * hx
        lm = loss(c["eps"], c["sigma"], p)
        fd = (lp - lm) / (2 * hx)
        assert abs(fd - gp[k, ax].item()) <= 1e-4 * max(1.0, abs(gp[k, ax].item())) + 4 * noise / hx
    m.bin(pos, sp, outputs=False)


def test_gradcheck_fp64():
    c = _two_species_small(4, n=2, hexes=2, rc=1.6)
    m = Mesh(c["mesh"], c["box"])
    m.build_lists(c["rc"], 1e-3)
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda", requires_grad=True)
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    eps = torch.tensor(c["eps"], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(c["sigma"], dtype=torch.float64, requires_grad=True)
    f = lambda p, e, s: LJForce.apply(p, e, s, m, sp, "fp64")
    # forces are summed with atomics, so repeated backward calls differ in the last bits
    assert torch.autograd.gradcheck(f, (pos, eps, sig), eps=1e-6, atol=1e-6, rtol=1e-5, nondet_tol=1e-12)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("S", [3, 8])
def test_vjp_up_to_eight_species(S, prec, tol):
    c = _two_species_small(5 + S)
    rng = np.random.default_rng(S)
    c["species"] = rng.integers(0, S, len(c["pos"])).astype(np.int32)
    c["eps"] = np.linspace(0.8, 1.6, S)
    c["sigma"] = np.linspace(0.9, 1.1, S)
    m, *_ = gpu_setup(c)
    v = rng.normal(size=c["pos"].shape)
    gx, ge, gs, _ = torch_ref.vjp(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], v)
    dt = torch.float64 if prec == "fp64" else torch.float32
    gp, ge_g, gs_g = m.forces_backward(c["eps"], c["sigma"], torch.tensor(v, dtype=dt, device="cuda"), prec)
    assert np.abs(gp.double().cpu().numpy() - gx).max() <= tol * np.abs(gx).max()
    np.testing.assert_allclose(ge_g.cpu().numpy(), ge, rtol=tol, atol=tol * np.abs(ge).max())
    np.testing.assert_allclose(gs_g.cpu().numpy(), gs, rtol=tol, atol=tol * np.abs(gs).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("S", [1, 2])
def test_wedge_adjoint_matches_image_reference(S, prec, tol):
    """General referring transforms: referred pairs are one-sided and the
    source molecule's gradient is rotated back."""
    from oracle import transforms as T
    c = synth.wedge(3)
    rng = np.random.default_rng(11)
    sp = rng.integers(0, S, len(c["pos"])).astype(np.int32)
    eps, sig = np.linspace(1.0, 1.5, S), np.linspace(1.0, 0.88, S)
    m = Mesh(c["mesh"], c["box"])
    m.set_transforms(c["transforms"])
    m.build_lists(c["rc"], c["skin"])
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    m.bin(pos, torch.tensor(sp, dtype=torch.int32, device="cuda"))
    v = rng.normal(size=c["pos"].shape)
    gx, ge, gs, _ = torch_ref.image_vjp(c["pos"], sp, eps, sig, c["rc"], T.closure(c["transforms"], 6), v)
    dt = torch.float64 if prec == "fp64" else torch.float32
    gp, ge_g, gs_g = m.forces_backward(eps, sig, torch.tensor(v, dtype=dt, device="cuda"), prec)
    assert np.abs(gp.double().cpu().numpy() - gx).max() <= tol * np.abs(gx).max()
    np.testing.assert_allclose(ge_g.cpu().numpy(), ge, rtol=tol, atol=tol * np.abs(ge).max())
    np.testing.assert_allclose(gs_g.cpu().numpy(), gs, rtol=tol, atol=tol * np.abs(gs).max())
    m.close()


@pytest.mark.parametrize("cfg", ["c2", "c4"])
def test_adjoint_full_size_sampled_rows(cfg):
    """At the full c2 / c4 sizes: sampled rows of dL/dx against the oracle's
    per-row gradient (both precisions), and the FP32 species sums against the
    FP64 ones (pinned against the oracle at small sizes above)."""
    c = synth.make(cfg, 0)
    m, *_ = gpu_setup(c)
    rng = np.random.default_rng(4)
    v = rng.normal(size=c["pos"].shape)
    idx = rng.choice(len(c["pos"]), 64, replace=False)
    ref = torch_ref.vjp_rows(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], v, idx)
    vd = torch.tensor(v, device="cuda")
    g64, ge64, gs64 = m.forces_backward(c["eps"], c["sigma"], vd, "fp64")
    g32, ge32, gs32 = m.forces_backward(c["eps"], c["sigma"], vd.float(), "fp32")
    scale = np.abs(ref).max()
    assert np.abs(g64.cpu().numpy()[idx] - ref).max() <= 1e-10 * scale
    assert np.abs(g32.double().cpu().numpy()[idx] - ref).max() <= 2e-4 * scale
    np.testing.assert_allclose(ge32.cpu().numpy(), ge64.cpu().numpy(), rtol=1e-4)
    np.testing.assert_allclose(gs32.cpu().numpy(), gs64.cpu().numpy(), rtol=1e-4)
