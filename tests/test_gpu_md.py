"""GPU velocity-Verlet against the FP64 oracle integrator."""
import numpy as np
import pytest
import torch

import synth
from oracle import md as omd
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


def test_md_c1_matches_oracle(mp):
    s, d = synth.cu_fcc_small(), synth.model_c1()
    w = synth.make_weights(d, 0)
    v0 = synth.maxwell(s.masses, 600.0, 4)
    n_steps, dt = 10, 1.0

    def force(p):
        e = onb.edges(p, s.box, d.r_cut)
        E, _, F = om.energy_forces(p, s.species, s.box, e, w, d, 2)
        return E, F

    pr, vr, _, led_r = omd.verlet(s.pos, v0, s.masses, s.box, force, dt, n_steps)
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    vel = torch.tensor(v0, device="cuda")
    frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
    mass = torch.tensor(s.masses, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    led = mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, dt, n_steps, n_layers=2)
    torch.cuda.synchronize()
    p = pos.cpu().numpy()
    dp = p - pr
    dp -= s.box * np.round(dp / s.box)
    assert np.abs(dp).max() < 1e-7
    assert np.abs(vel.cpu().numpy() - vr).max() < 1e-7
    assert np.abs(led - led_r).max() < 1e-5 * np.abs(led_r[:, 2]).max()
    pot.close()


def test_md_partitioned_equals_unpartitioned_and_conserves(mp):
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.05, seed=2)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 300.0, 5)
    out = []
    for parts in (1, 4):
        pot = mp.Potential(d, w)
        pos = torch.tensor(s.pos, device="cuda")
        vel = torch.tensor(v0, device="cuda")
        frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
        led = mp.mp_md_step(pot.ctx, pos, vel, frc, torch.tensor(s.masses, device="cuda"),
                            torch.tensor(s.species, device="cuda"), s.box, 0.5, 20, n_layers=2,
                            n_parts=parts, k_hops=2)
        out.append((pos.cpu().numpy(), led))
        pot.close()
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-6
    led = out[0][1]
    # NVE: total energy fluctuation small compared with the kinetic energy
    assert np.ptp(led[:, 2]) < 1e-2 * led[:, 1].mean()
