"""Pins of the oracle's BAOAB Langevin integrator."""
import math

import numpy as np

import synth
from oracle import md as omd


def _harmonic(k):
    def force(p):
        return 0.5 * k * float((p * p).sum()), -k * p
    return force


def test_zero_friction_is_velocity_verlet():
    rng = np.random.default_rng(0)
    m = rng.uniform(20, 60, 50)
    x0, v0 = rng.normal(0, 0.1, (50, 3)), rng.normal(0, 0.01, (50, 3))
    f = _harmonic(2.0)
    xa, va, _, la = omd.langevin(x0, v0, m, None, f, 1.0, 30, T=300.0, gamma=0.0, seed=1)
    xb, vb, _, lb = omd.verlet(x0, v0, m, None, f, 1.0, 30)
    assert np.abs(xa - xb).max() < 1e-12 and np.abs(va - vb).max() < 1e-13


def test_harmonic_configurational_temperature():
    # BAOAB samples the configurational distribution of a harmonic oscillator
    # exactly (below the stability limit): <k x^2> = kB T per component.
    n, T, k = 4000, 400.0, 5.0
    m = np.full(n, 30.0)
    f = _harmonic(k)
    x, v = np.zeros((n, 3)), np.zeros((n, 3))
    x, v, _, _ = omd.langevin(x, v, m, None, f, 2.0, 300, T=T, gamma=0.05, seed=7)
    samples = []
    for blk in range(20):
        x, v, _, _ = omd.langevin(x, v, m, None, f, 2.0, 20, T=T, gamma=0.05, seed=7,
                                  step0=300 + 20 * blk)
        samples.append(k * (x * x).mean())
    kt = synth.KB_EV * T
    assert abs(np.mean(samples) / kt - 1) < 0.02


def test_noise_counters():
    # step s, atom i, axis a uses counter (s N + i) 3 + a of the Langevin stream
    xi = synth.normal_at(5, synth.STREAM_LANGEVIN, np.arange(12, dtype=np.uint64))
    assert np.array_equal(xi, synth.normal(5, synth.STREAM_LANGEVIN, 12))
    assert abs(xi.mean()) < 2 and 0.2 < xi.std() < 3
