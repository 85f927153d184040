"""Pins for the oracle's velocity-Verlet integrator (CPU only): free flight,
second-order energy error, time reversibility, momentum conservation."""
import numpy as np

import oracle
from paper_cs_0702131_gb300 import synth

BIG = dict(L=np.array([40.0, 40.0, 40.0]), periodic=np.array([1, 1, 1], np.int32))
ONE = (np.array([1.0]), np.array([1.0]))


def test_free_flight_is_linear():
    pos = np.array([[5.0, 5.0, 5.0], [20.0, 20.0, 20.0]])
    vel = np.array([[0.3, -0.2, 0.1], [-0.1, 0.05, 0.4]])
    sp = np.zeros(2, np.int32)
    r = oracle.verlet(pos, vel, sp, *ONE, [2.0], 2.5, BIG, 0.01, 50)
    np.testing.assert_allclose(r["pos"], pos + 50 * 0.01 * vel, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["vel"], vel)
    np.testing.assert_allclose(r["KE"], r["KE"][0], rtol=1e-15)


def _dimer(dt, T=1.0):
    pos = np.array([[10.0, 10.0, 10.0], [11.2, 10.1, 10.0]])
    vel = np.array([[0.5, 0.2, 0.0], [-0.5, -0.2, 0.1]])
    r = oracle.verlet(pos, vel, np.zeros(2, np.int32), *ONE, [1.0], 2.5, BIG, dt, int(round(T / dt)))
    E = r["KE"] + r["PE"]
    return np.abs(E - E[0]).max()


def test_energy_error_is_second_order():
    e1, e2 = _dimer(0.002), _dimer(0.001)
    assert 3.0 < e1 / e2 < 5.0


def test_time_reversible_and_momentum_conserving():
    c = synth.make("t0", 1)
    rng = np.random.default_rng(5)
    v0 = rng.normal(scale=0.5, size=c["pos"].shape)
    mass = [1.0]
    f = oracle.verlet(c["pos"], v0, c["species"], c["eps"], c["sigma"], mass, c["rc"], c["box"], 0.002, 20)
    b = oracle.verlet(f["pos"], -f["vel"], c["species"], c["eps"], c["sigma"], mass, c["rc"], c["box"], 0.002, 20)
    np.testing.assert_allclose(b["pos"], c["pos"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(-b["vel"], v0, rtol=0, atol=1e-9)
    scale = np.abs(v0).sum()
    assert np.abs(f["P"] - f["P"][0]).max() <= 1e-12 * scale
