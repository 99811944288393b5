"""Verlet-skin reuse of neighbours and partitions in mp_md_step: the list is
built with r_c + skin (halos in units of r_c + skin) and kept until some atom
has moved more than skin / 2, and its pairs beyond r_c add exact zeros.  So
a skin run follows the run that rebuilds every step (to FP32 summation
order: the two lists hold the same pairs within r_c in another order), and
the forces it ends with, from a list built steps earlier, equal a fresh
evaluation at its final positions."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _setup(mp):
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.08, seed=7)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 900.0, 8)
    return s, d, w, v0


def _run(mp, pot, s, v0, steps, **kw):
    dev = torch.device("cuda")
    pos = torch.tensor(s.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device=dev)
    mass = torch.tensor(s.masses, device=dev)
    sp = torch.tensor(s.species, device=dev)
    builds = []
    led = mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, 1.0, steps, builds=builds, **kw)
    torch.cuda.synchronize()
    return pos, vel, frc, led, builds[0]


@pytest.mark.parametrize("precision,parts,mode", [("fp32", 1, 0), ("fp32", 4, 0),
                                                  ("fp32", 4, 1), ("bf16", 4, 0)])
def test_skin_run_follows_rebuilt_run_and_reused_list_is_exact(mp, precision, parts, mode):
    s, d, w, v0 = _setup(mp)
    prec = mp.MP_FP32 if precision == "fp32" else mp.MP_BF16
    md = dict(n_layers=2, precision=prec, n_parts=parts, k_hops=2, halo_mode=mode)
    steps = 30
    pot = mp.Potential(d, w)
    try:
        p0, v_0, f0, led0, b0 = _run(mp, pot, s, v0, steps, **md)
        p1, v_1, f1, led1, b1 = _run(mp, pot, s, v0, steps, skin=0.8, **md)
        assert b0 == steps + 1            # the initial forces and every step
        assert 1 <= b1 < steps // 3       # reused for several steps at a time
        L = torch.tensor(s.box, device="cuda", dtype=torch.float64)
        wrap = lambda p: p - L * torch.floor(p / L)
        dp = wrap(p1) - wrap(p0)
        dp = dp - L * torch.round(dp / L)
        tol_x = 1e-5 if precision == "bf16" else 1e-6
        assert float(dp.abs().max()) <= tol_x
        assert np.allclose(led1, led0, rtol=1e-6, atol=1e-6 * len(s.pos))
        # the skin run's last forces came from a list built steps before
        # (positions may lie outside the box by less than skin / 2)
        E, F, _ = pot.energy_forces(p1, torch.tensor(s.species, device="cuda"), s.box, 2, prec,
                                    n_parts=parts, halo_mode=mode)
        torch.cuda.synchronize()
        a, b = F.cpu().numpy().astype(np.float64), f1.cpu().numpy().astype(np.float64)
        frms = np.sqrt((a ** 2).mean())
        tol_f = 1e-4 if precision == "bf16" else 2e-6
        assert np.abs(b - a).max() <= tol_f * frms, np.abs(b - a).max() / frms
        assert abs(led1[-1, 0] - float(E.item())) <= 1e-6 * abs(float(E.item()))
    finally:
        pot.close()


def test_list_kept_across_calls_and_rebuilt_after_a_large_move(mp):
    s, d, w, v0 = _setup(mp)
    md = dict(n_layers=2, precision=mp.MP_FP32, n_parts=4, k_hops=2, halo_mode=0, skin=1.0)
    pot = mp.Potential(d, w)
    dev = torch.device("cuda")
    try:
        pos = torch.tensor(s.pos, device=dev)
        vel = torch.tensor(v0, device=dev)
        frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device=dev)
        mass = torch.tensor(s.masses, device=dev)
        sp = torch.tensor(s.species, device=dev)
        nb = []
        mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, 1.0, 2, builds=nb, **md)
        mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, 1.0, 2, forces_valid=True,
                      builds=nb, **md)
        assert nb == [1, 0]               # the second call continues on the first's list
        pos[5] += torch.tensor([0.7, 0.0, 0.0], device=dev, dtype=torch.float64)
        mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, 1.0, 1, builds=nb, **md)
        assert nb[-1] >= 1                # an atom moved by more than skin / 2
        E, F, _ = pot.energy_forces(pos, sp, s.box, 2, mp.MP_FP32, n_parts=4)
        torch.cuda.synchronize()
        a, b = F.cpu().numpy().astype(np.float64), frc.cpu().numpy().astype(np.float64)
        assert np.abs(b - a).max() <= 2e-6 * np.sqrt((a ** 2).mean())
        with pytest.raises(mp.MPError) as e:
            mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, 1.0, 1,
                          **dict(md, skin=-0.5))
        assert e.value.code == mp.MP_ERR_ARG
    finally:
        pot.close()
