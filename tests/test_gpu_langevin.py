"""GPU BAOAB Langevin dynamics against the FP64 oracle integrator."""
import numpy as np
import pytest
import torch

import synth
from oracle import md as omd
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


def _run(mp, s, d, w, v0, n_steps, dt, K, T, gamma, seed, step0=0, pot=None, state=None,
         forces_valid=False):
    own = pot is None
    if own:
        pot = mp.Potential(d, w)
    if state is None:
        state = (torch.tensor(s.pos, device="cuda"), torch.tensor(v0, device="cuda"),
                 torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda"))
    pos, vel, frc = state
    led = mp.mp_md_step(pot.ctx, pos, vel, frc, torch.tensor(s.masses, device="cuda"),
                        torch.tensor(s.species, device="cuda"), s.box, dt, n_steps, n_layers=K,
                        thermostat=mp.MP_LANGEVIN, temperature=T, friction=gamma, seed=seed,
                        step0=step0, forces_valid=forces_valid)
    torch.cuda.synchronize()
    if own:
        pot.close()
    return pos.cpu().numpy(), vel.cpu().numpy(), led


def _oracle(s, d, w, v0, n_steps, dt, K, T, gamma, seed):
    def force(p):
        E, _, F = om.energy_forces(p, s.species, s.box, onb.edges(p, s.box, d.r_cut), w, d, K)
        return E, F
    return omd.langevin(s.pos, v0, s.masses, s.box, force, dt, n_steps, T, gamma, seed)


def _dpos(p, q, box):
    dp = p - q
    return np.abs(dp - box * np.round(dp / box)).max()


def test_force_free_steps_match_oracle(mp):
    # K = 0 and no pair term: F = 0, so every difference would come from the
    # integrator or the noise generator (counters, splitmix64, Box-Muller).
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.05, seed=3)
    d = synth.model_alloy(n_layers_full=1)
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 600.0, 9)
    p, v, _ = _run(mp, s, d, w, v0, 6, 1.0, 0, 600.0, 0.02, 1234)
    pr, vr, _, _ = _oracle(s, d, w, v0, 6, 1.0, 0, 600.0, 0.02, 1234)
    assert _dpos(p, pr, s.box) < 1e-12
    assert np.abs(v - vr).max() < 1e-13


def test_steps_with_forces_match_oracle(mp):
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.05, seed=3)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 600.0, 9)
    p, v, led = _run(mp, s, d, w, v0, 5, 1.0, 2, 600.0, 0.02, 77)
    pr, vr, _, led_r = _oracle(s, d, w, v0, 5, 1.0, 2, 600.0, 0.02, 77)
    assert _dpos(p, pr, s.box) < 1e-7
    assert np.abs(v - vr).max() < 1e-7
    assert np.abs(led - led_r).max() < 1e-5 * np.abs(led_r[:, 2]).max()


def test_continued_run_equals_single_run(mp):
    # step0 carries the noise counters across calls; the context keeps its
    # buffers between calls: 3 + 3 steps equal 6 steps bit for bit.
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.05, seed=3)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 500.0, 2)
    p6, v6, _ = _run(mp, s, d, w, v0, 6, 1.0, 2, 500.0, 0.05, 5)
    pot = mp.Potential(d, w)
    state = (torch.tensor(s.pos, device="cuda"), torch.tensor(v0, device="cuda"),
             torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda"))
    _run(mp, s, d, w, v0, 3, 1.0, 2, 500.0, 0.05, 5, pot=pot, state=state)
    p3, v3, _ = _run(mp, s, d, w, v0, 3, 1.0, 2, 500.0, 0.05, 5, step0=3, pot=pot, state=state,
                     forces_valid=True)
    pot.close()
    assert np.array_equal(p6, p3) and np.array_equal(v6, v3)


def test_thermostat_reaches_target_temperature(mp):
    # 864 atoms from rest, T = 800 K, gamma = 0.05 / fs: the kinetic
    # temperature over the last 200 of 400 steps averages to T within 10 %.
    s = synth.alloy_fcc(cells=(6, 6, 6), sigma=0.05, seed=3)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    n = len(s.pos)
    _, _, led = _run(mp, s, d, w, np.zeros((n, 3)), 400, 1.0, 2, 800.0, 0.05, 11)
    t_kin = 2.0 * led[200:, 1] / (3 * n * synth.KB_EV)
    assert abs(t_kin.mean() / 800.0 - 1.0) < 0.10, t_kin.mean()
