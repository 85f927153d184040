"""Pins for the oracle's all-pairs LJ sum (CPU only).

Closed forms (two and three molecules, perfect-FCC lattice sums), Newton's
third law, F = -grad U by central differences, the minimum image across a
periodic boundary, the energy shift and the mixing rule.
"""
import numpy as np
import pytest

import oracle
from paper_cs_0702131_gb300 import synth
from conftest import big_box


def _lj(pos, rc=2.5, box=None, species=None, eps=(1.0,), sigma=(1.0,), shift=False):
    pos = np.asarray(pos, dtype=np.float64)
    sp = np.zeros(len(pos), np.int32) if species is None else np.asarray(species, np.int32)
    return oracle.lj(pos, sp, np.asarray(eps), np.asarray(sigma), rc, box or big_box(), shift=shift)


def test_two_molecules(golden):
    rng = np.random.default_rng(1)
    for row in golden["two_molecule"]:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x0 = np.array([50.0, 50.0, 50.0])
        pos = [x0, x0 - row["r"] * d]          # d points from molecule 1 to molecule 0
        r = _lj(pos, rc=3.5)
        assert r["pairs"] == 1
        np.testing.assert_allclose(r["U"], row["u"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["F"][0], row["f"] * d, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(r["F"][1], -row["f"] * d, rtol=1e-11, atol=1e-12)
        # virial of one pair: W_ab = r_a f_b, trace = r f
        np.testing.assert_allclose(r["W"][:3].sum(), row["r"] * row["f"], rtol=1e-11, atol=1e-12)


def test_cutoff_is_strict_and_truncated():
    x0 = np.array([50.0, 50.0, 50.0])
    inside = _lj([x0, x0 + [2.5 - 1e-9, 0, 0]], rc=2.5)
    outside = _lj([x0, x0 + [2.5 + 1e-9, 0, 0]], rc=2.5)
    assert inside["pairs"] == 1 and outside["pairs"] == 0
    assert outside["U"] == 0.0 and np.all(outside["F"] == 0)


def test_three_molecules(golden):
    eq = golden["equilateral_side_1"]
    P = np.array([[0, 0, 0], [1, 0, 0], [0.5, np.sqrt(3) / 2, 0]]) + 40.0
    r = _lj(P)
    ctr = P.mean(0)
    for k in range(3):
        out = (P[k] - ctr) / np.linalg.norm(P[k] - ctr)
        np.testing.assert_allclose(r["F"][k], eq["net_force"] * out, rtol=1e-12, atol=1e-12)
    assert abs(r["U"]) < 1e-12
    col = golden["collinear_minimum"]
    s = col["spacing"]
    P = np.array([[0, 0, 0], [s, 0, 0], [2 * s, 0, 0]]) + 40.0
    r = _lj(P)
    np.testing.assert_allclose(r["U"], col["U"], rtol=1e-12)
    np.testing.assert_allclose(r["F"][0, 0], -col["end_force"], rtol=1e-9)   # end pair pulls inward
    np.testing.assert_allclose(r["F"][2, 0], col["end_force"], rtol=1e-9)
    assert abs(r["F"][1]).max() < 1e-12


@pytest.mark.parametrize("rc", ["2.5", "3"])
def test_perfect_fcc_lattice_sums(golden, rc):
    g = golden["fcc_rho08"]
    a = g["a"]
    pos = synth.fcc_sites(6, 6, 6, a)
    L = 6 * a
    box = dict(L=np.array([L, L, L]), periodic=np.array([1, 1, 1], np.int32))
    r = _lj(pos, rc=float(rc), box=box)
    n = len(pos)
    assert r["pairs"] == g[rc]["pairs_per_N"] * n
    np.testing.assert_allclose(r["U"] / n, g[rc]["U_per_N"], rtol=1e-11)
    np.testing.assert_allclose(r["W"][:3].sum() / n, g[rc]["virial_rf_per_N"], rtol=1e-11)
    assert np.abs(r["F"]).max() < 1e-11                  # every site is a centre of symmetry
    np.testing.assert_allclose(r["W"][3:], 0, atol=1e-9)   # cubic symmetry: no shear


@pytest.mark.parametrize("name", ["c1", "t0"])
def test_newton_third_law(name):
    c = synth.make(name, seed=3)
    r = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    assert np.abs(r["F"].sum(0)).max() <= 1e-12 * r["Fabs"].sum()


def test_force_is_minus_gradient_of_energy():
    c = synth.make("c1", seed=5)
    pos, box = c["pos"], c["box"]
    h = 1e-5
    rng = np.random.default_rng(0)
    r0 = oracle.lj(pos, c["species"], c["eps"], c["sigma"], c["rc"], box)
    checked = 0
    for k in rng.permutation(len(pos)):
        d = pos - pos[k]
        d -= box["L"] * np.round(d / box["L"])
        rr = np.linalg.norm(d, axis=1)
        if np.any(np.abs(rr - c["rc"]) < 10 * h):
            continue                                     # the truncation step is not differentiable
        for ax in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, ax] += h
            pm[k, ax] -= h
            Up = oracle.lj(pp, c["species"], c["eps"], c["sigma"], c["rc"], box)["U"]
            Um = oracle.lj(pm, c["species"], c["eps"], c["sigma"], c["rc"], box)["U"]
            fd = -(Up - Um) / (2 * h)
            assert abs(fd - r0["F"][k, ax]) <= 1e-6 * max(1.0, r0["Fabs"][k])
        checked += 1
        if checked == 6:
            break
    assert checked == 6


def test_minimum_image_across_boundary():
    box = dict(L=np.array([10.0, 10.0, 10.0]), periodic=np.array([1, 1, 1], np.int32))
    r = _lj([[0.1, 5, 5], [9.0, 5, 5]], box=box)        # 1.1 apart through x = 0
    assert r["pairs"] == 1
    f = 24 * (2 * 1.1 ** -13 - 1.1 ** -7)
    np.testing.assert_allclose(r["F"][0], [f, 0, 0], rtol=1e-12)
    box["periodic"] = np.array([0, 1, 1], np.int32)       # same pair, x not periodic: 8.9 apart
    assert _lj([[0.1, 5, 5], [9.0, 5, 5]], box=box)["pairs"] == 0


def test_energy_shift_moves_each_pair_by_u_rc(golden):
    c = synth.make("c1", seed=2)
    a = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    b = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], shift=True)
    u_rc = [row["u"] for row in golden["two_molecule"] if row["what"] == "2.5"][0]
    np.testing.assert_allclose(b["U"], a["U"] - a["pairs"] * u_rc, rtol=1e-12)
    np.testing.assert_array_equal(a["F"], b["F"])


def test_lorentz_berthelot_mixing():
    # species 0: sigma 1, eps 1; species 1: sigma 0.88, eps 1.5.  The unlike pair
    # has its minimum at 2^(1/6) * 0.94 with depth sqrt(1.5).
    x0 = np.array([30.0, 30.0, 30.0])
    rmin = 2 ** (1 / 6) * 0.94
    r = _lj([x0, x0 + [rmin, 0, 0]], species=[0, 1], eps=(1.0, 1.5), sigma=(1.0, 0.88))
    np.testing.assert_allclose(r["U"], -np.sqrt(1.5), rtol=1e-12)
    assert np.abs(r["F"]).max() < 1e-12
    r = _lj([x0, x0 + [0.94, 0, 0]], species=[0, 1], eps=(1.0, 1.5), sigma=(1.0, 0.88))
    np.testing.assert_allclose(r["F"][0, 0], -24 * np.sqrt(1.5) / 0.94, rtol=1e-12)


def test_sampled_rows_equal_full():
    c = synth.make("t0", seed=1)
    full = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    idx = np.array([0, 5, 17, 400, 863])
    part = oracle.lj(c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"], idx=idx)
    np.testing.assert_array_equal(part["F"], full["F"][idx])


@pytest.mark.parametrize("name", ["t0", "h0", "c1", "c4", "slab"])
def test_cubic_cell_baseline_equals_all_pairs(name):
    """The cubic-cell baseline (§2.1) visits exactly the pairs within rc."""
    if name == "slab":
        c = synth.nanochannel(3, nfcc=(12, 4, 12), hex_shape=(8, 4, 8), post_radius=2.0)
    else:
        c = synth.make(name, seed=4)
    args = (c["pos"], c["species"], c["eps"], c["sigma"], c["rc"], c["box"])
    a = oracle.lj(*args)
    b = oracle.lj_cells(*args)
    assert a["row_pairs"] == b["row_pairs"]
    scale = a["Fabs"][:, None] + 1e-300
    assert np.max(np.abs(a["F"] - b["F"]) / scale) < 1e-13
    assert abs(a["U"] - b["U"]) <= 1e-13 * a["Uabs"]
    assert np.all(np.abs(a["W"] - b["W"]) <= 1e-13 * a["Wabs"])
