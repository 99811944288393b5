"""Correction-head workflow on the GPU (the learned part).

1. Snapshots from the method's own MD: NVE runs of the pruned (K-layer)
   model on binary-alloy FCC cells, started from Maxwell velocities at
   temperatures spread over a range; snapshots every `every` steps after an
   equilibration.
2. Labels: energies and forces of the full-depth model on each snapshot.
3. Training: Adam on the head parameters with the library's loss/gradient
   kernels (backbone frozen), one snapshot per step.
4. Judgement: force RMSE against the full-depth model on held-out snapshots
   and on larger cells, for the pruned model alone and with the head; and
   MD in which the full-depth model checks the student every `check_every`
   steps and replaces its forces when the student's error exceeds twice the
   validation RMSE.

Every computation runs through the C ABI of libmpip.so.

    python -m paper_2509_21694_gb300.head_train [--runs 20 --snaps 100 ...]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import synth
from . import binding as mp


def make_potential(layers_full: int = 6, rep_eps: float = 0.3, seed: int = 1):
    d = synth.model_alloy(n_layers_full=layers_full)
    d.rep_eps = rep_eps
    return mp.Potential(d, synth.make_weights(d, seed)), d


def generate(pot, K, runs=20, snaps=100, every=20, equil=200, cells=(6, 6, 6),
             t_lo=300.0, t_hi=1500.0, dt=1.0, seed=3):
    """List of snapshots (pos, species, box, E_teacher, F_teacher, E_pruned, F_pruned)."""
    out = []
    L_full = pot.desc.n_layers_full
    for r in range(runs):
        T = t_lo + (t_hi - t_lo) * (r / max(1, runs - 1))
        s = synth.alloy_fcc(cells=cells, sigma=0.05, seed=seed * 1000 + r)
        pos = torch.tensor(s.pos, device="cuda")
        vel = torch.tensor(synth.maxwell(s.masses, T, seed * 1000 + r), device="cuda")
        frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
        mass = torch.tensor(s.masses, device="cuda")
        sp = torch.tensor(s.species, device="cuda")
        md = dict(n_layers=K, ledger=False)
        mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, dt, equil, **md)
        for k in range(snaps):
            mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, dt, every, forces_valid=True, **md)
            Et, Ft, _ = pot.energy_forces(pos, sp, s.box, L_full)
            Ep, Fp, _ = pot.energy_forces(pos, sp, s.box, K)
            out.append((pos.clone(), sp, s.box, Et.clone(), Ft.clone(), Ep.clone(), Fp.clone()))
    return out


def force_rmse(pot, snaps, K, use_head):
    err, n = 0.0, 0
    for pos, sp, box, Et, Ft, _, _ in snaps:
        _, F, _ = pot.energy_forces(pos, sp, box, K, use_head=use_head)
        err += ((F.double() - Ft.double()) ** 2).sum().item()
        n += F.numel()
    return float(np.sqrt(err / n))


def train(pot, K, snaps, epochs=20, lr=1e-3, lam=1.0, seed=0):
    rng = np.random.default_rng(seed)
    step = 0
    hist = []
    for ep in range(epochs):
        tot = 0.0
        for q in rng.permutation(len(snaps)):
            pos, sp, box, Et, Ft, _, _ = snaps[q]
            g = mp.mp_build_neighbors(pot.ctx, pos, box)
            try:
                loss, grad = mp.mp_head_loss_grad(pot.ctx, pos, sp, g, K, Et, Ft, lam)
                step += 1
                mp.mp_head_adam_step(pot.ctx, grad, lr, step)
                tot += loss.item()
            finally:
                mp.mp_graph_free(g)
        hist.append(tot / len(snaps))
    return hist


def judged_md(pot, K, cells, T, steps, check_every, threshold, dt=1.0, seed=11):
    """Student MD with the full-depth model as judge and fallback."""
    L_full = pot.desc.n_layers_full
    s = synth.alloy_fcc(cells=cells, sigma=0.05, seed=seed)
    pos = torch.tensor(s.pos, device="cuda")
    vel = torch.tensor(synth.maxwell(s.masses, T, seed), device="cuda")
    frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
    mass = torch.tensor(s.masses, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    checks, fallbacks, errs = 0, 0, []
    done = 0
    while done < steps:
        n = min(check_every, steps - done)
        mp.mp_md_step(pot.ctx, pos, vel, frc, mass, sp, s.box, dt, n, n_layers=K, use_head=True,
                      forces_valid=done > 0, ledger=False)
        done += n
        _, Ft, _ = pot.energy_forces(pos, sp, s.box, L_full)
        e = torch.sqrt(((frc.double() - Ft.double()) ** 2).mean()).item()
        errs.append(e)
        checks += 1
        if e > threshold:
            frc.copy_(Ft)          # the judge's forces replace the student's for the next step
            fallbacks += 1
    return {"atoms": len(s.pos), "steps": steps, "checks": checks, "fallbacks": fallbacks,
            "student_force_rmse_at_checks": errs}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--snaps", type=int, default=100)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--equil", type=int, default=200)
    ap.add_argument("--cells", type=int, default=6)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--val", type=float, default=0.1)
    ap.add_argument("--eval-cells", type=int, default=20)
    ap.add_argument("--md-steps", type=int, default=200)
    args = ap.parse_args(argv)
    K = 2
    pot, d = make_potential()
    t0 = time.time()
    snaps = generate(pot, K, args.runs, args.snaps, args.every, args.equil, (args.cells,) * 3)
    t_gen = time.time() - t0
    rng = np.random.default_rng(0)
    order = rng.permutation(len(snaps))
    n_val = max(1, int(round(args.val * len(snaps))))
    val = [snaps[q] for q in order[:n_val]]
    trn = [snaps[q] for q in order[n_val:]]
    # start from a zero-output head so the untrained student equals the pruned model
    h = mp.mp_head_get(pot.ctx)
    h[32 * d.F + 32:] = 0.0
    mp.mp_set_head(pot.ctx, h)
    before = force_rmse(pot, val, K, use_head=False)
    t0 = time.time()
    hist = train(pot, K, trn, args.epochs, args.lr)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    after = force_rmse(pot, val, K, use_head=True)
    big = generate(pot, K, runs=2, snaps=1, every=20, equil=50, cells=(args.eval_cells,) * 3,
                   t_lo=600.0, t_hi=1200.0, seed=9)
    out = {
        "snapshots": len(snaps), "atoms_per_snapshot": 4 * args.cells ** 3,
        "label_generation_s": t_gen, "train_steps": len(trn) * args.epochs,
        "train_s": t_train, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
        "val_force_rmse_pruned": before, "val_force_rmse_student": after,
        "eval_atoms": 4 * args.eval_cells ** 3,
        "eval_force_rmse_pruned": force_rmse(pot, big, K, use_head=False),
        "eval_force_rmse_student": force_rmse(pot, big, K, use_head=True),
    }
    out["judged_md"] = judged_md(pot, K, (args.eval_cells,) * 3, 900.0, args.md_steps, 100,
                                 2.0 * after)
    print(json.dumps(out))
    pot.close()
    return out


if __name__ == "__main__":
    main()
