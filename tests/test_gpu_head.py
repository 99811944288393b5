"""Correction head (the learned part) on the GPU: inference and the loss
gradient (forward-mode tangent pass + per-atom terms) against the FP64
oracle, and training gains against the full-depth teacher."""
import numpy as np
import pytest
import torch

import synth
from oracle import head as oh
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


def _snapshot(seed=4, cells=(4, 4, 4)):
    s = synth.alloy_fcc(cells=cells, sigma=0.1, seed=seed)
    d = synth.model_alloy(n_layers_full=6)
    w = synth.make_weights(d, 1)
    return s, d, w


def test_head_inference_fp32(mp):
    s, d, w = _snapshot()
    pot = mp.Potential(d, w)
    E, F, _ = pot.energy_forces(torch.tensor(s.pos, device="cuda"),
                                torch.tensor(s.species, device="cuda"), s.box, 2, use_head=True)
    Er, Eir, Fr = om.energy_forces(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w,
                                   d, 2, use_head=True)
    frms = np.sqrt((Fr ** 2).mean())
    assert np.abs(F.cpu().numpy() - Fr).max() <= 1e-5 * frms
    assert abs(E.item() - Er) <= 1e-6 * len(s.pos) * np.sqrt((Eir ** 2).mean())
    pot.close()


@pytest.mark.parametrize("lam,K", [(1.0, 2), (0.0, 2), (1.0, 1)])
def test_head_loss_gradient_matches_oracle(mp, lam, K):
    s, d, w = _snapshot(seed=6)
    rng = np.random.default_rng(3)
    e_ref = 1.02 * om.energy(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w, d, K)
    f_ref = rng.normal(0, 0.4, s.pos.shape)
    Lr, gr = oh.loss_and_grad(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w, d, K,
                              e_ref, f_ref, lam)
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    try:
        loss, grad = mp.mp_head_loss_grad(
            pot.ctx, pos, torch.tensor(s.species, device="cuda"), g, K,
            torch.tensor([e_ref], dtype=torch.float64, device="cuda"),
            torch.tensor(f_ref, dtype=torch.float32, device="cuda"), lam)
        torch.cuda.synchronize()
        L = loss.item()
        G = grad.cpu().numpy()
    finally:
        mp.mp_graph_free(g)
        pot.close()
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    assert np.abs(G - gr).max() <= 1e-4 * np.abs(gr).max(), np.abs(G - gr).max() / np.abs(gr).max()


def test_head_training_beats_pruned_model(mp):
    # Teacher: the full 6-layer model; student: its first 2 layers + head.
    # Snapshots from short pruned-model MD of 256-atom alloy cells.
    d = synth.model_alloy(n_layers_full=6)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    pot = mp.Potential(d, w)
    snaps = []
    for k in range(6):
        s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.05, seed=20 + k)
        pos = torch.tensor(s.pos, device="cuda")
        vel = torch.tensor(synth.maxwell(s.masses, 300.0 + 200.0 * k, 30 + k), device="cuda")
        frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
        sp = torch.tensor(s.species, device="cuda")
        mp.mp_md_step(pot.ctx, pos, vel, frc, torch.tensor(s.masses, device="cuda"), sp, s.box,
                      1.0, 20, n_layers=2, ledger=False)
        Et, Ft, _ = pot.energy_forces(pos, sp, s.box, 6)
        Ep, Fp, _ = pot.energy_forces(pos, sp, s.box, 2)
        snaps.append((s, pos.clone(), sp, Et.clone(), Ft.clone(), Fp.clone()))
    train, held = snaps[:4], snaps[4:]

    def rmse(use_head):
        err = []
        for s, pos, sp, Et, Ft, Fp in held:
            _, F, _ = pot.energy_forces(pos, sp, s.box, 2, use_head=use_head)
            err.append(((F - Ft) ** 2).mean().item())
        return float(np.sqrt(np.mean(err)))

    # start from a zero-output head: the student equals the pruned model
    head0 = mp.mp_head_get(pot.ctx)
    n1 = 32 * 128 + 32
    head0[n1:] = 0.0
    mp.mp_set_head(pot.ctx, head0)
    base = rmse(False)
    assert abs(rmse(True) - base) < 1e-6 * base
    step = 0
    for epoch in range(40):
        for s, pos, sp, Et, Ft, Fp in train:
            g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
            _, grad = mp.mp_head_loss_grad(pot.ctx, pos, sp, g, 2, Et, Ft, 1.0)
            step += 1
            mp.mp_head_adam_step(pot.ctx, grad, 3e-3, step)
            mp.mp_graph_free(g)
    torch.cuda.synchronize()
    trained = rmse(True)
    pot.close()
    assert trained < 0.9 * base, (trained, base)
