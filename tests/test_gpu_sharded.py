"""The multi-GPU partition distribution's GPU pieces on one GPU: shares of
partition ranges (mp_energy_forces_parts) summed over ranges that cover the
plan equal the single call's energy and forces, and the sharded MD loop
(ranges evaluated in turn, the two Verlet halves through the C ABI) follows
mp_md_step's trajectory."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _setup(mp):
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.08, seed=5)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    pot = mp.Potential(d, w)
    return s, d, w, pot


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_partition_ranges_sum_to_the_single_call(mp, precision):
    s, d, w, pot = _setup(mp)
    prec = mp.MP_FP32 if precision == "fp32" else mp.MP_BF16
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    plan, _ = mp.mp_partition(pot.ctx, g, 4, 2, mp.MP_HALO_GEOM)
    try:
        E, F, e_atom = mp.mp_energy_forces(pot.ctx, pos, sp, g, plan, 2, prec,
                                           e_atom=torch.empty(len(s.pos), dtype=torch.float64,
                                                              device="cuda"))
        e_sum = torch.zeros(1, dtype=torch.float64, device="cuda")
        f_sum = torch.zeros(len(s.pos), 3, dtype=torch.float64, device="cuda")
        ea_sum = torch.zeros(len(s.pos), dtype=torch.float64, device="cuda")
        for b, e in ((0, 1), (1, 3), (3, 4)):
            ea = torch.full((len(s.pos),), 7.0, dtype=torch.float64, device="cuda")
            e_p, f_p, _ = mp.mp_energy_forces_parts(pot.ctx, pos, sp, g, plan, b, e, 2, prec,
                                                    e_atom=ea)
            e_sum += e_p
            f_sum += f_p
            ea_sum += ea
        # an empty range contributes nothing
        e0, f0, _ = mp.mp_energy_forces_parts(pot.ctx, pos, sp, g, plan, 2, 2, 2, prec)
        with pytest.raises(mp.MPError):
            mp.mp_energy_forces_parts(pot.ctx, pos, sp, g, plan, 3, 5, 2, prec)
        torch.cuda.synchronize()
        assert float(e0.item()) == 0.0 and float(f0.abs().max().item()) == 0.0
        E, F = float(E.item()), F.cpu().numpy().astype(np.float64)
        frms = np.sqrt((F ** 2).mean())
        assert abs(float(e_sum.item()) - E) <= 1e-12 * abs(E)
        # per-atom root energies: each atom is a root of exactly one range
        assert np.array_equal(ea_sum.cpu().numpy(), e_atom.cpu().numpy())
        # FP64 shares summed in another order, then rounded: one FP32 ulp at most
        f32 = f_sum.float().cpu().numpy().astype(np.float64)
        assert np.abs(f32 - F).max() <= 2.0 ** -22 * np.abs(F).max() + 1e-12 * frms
    finally:
        mp.mp_plan_free(plan)
        mp.mp_graph_free(g)
        pot.close()


def test_sharded_md_loop_follows_md_step(mp):
    from paper_2509_21694_gb300.sharded import LibraryOps, ShardedSystem
    s, d, w, pot = _setup(mp)
    dev = torch.device("cuda")
    sp = torch.tensor(s.species, device=dev)
    mass = torch.tensor(s.masses, device=dev)
    v0 = synth.maxwell(s.masses, 600.0, 4)
    # reference: the library's own MD loop, 4 slabs
    p_ref = torch.tensor(s.pos, device=dev)
    v_ref = torch.tensor(v0, device=dev)
    f_ref = torch.zeros(len(s.pos), 3, dtype=torch.float32, device=dev)
    led_ref = mp.mp_md_step(pot.ctx, p_ref, v_ref, f_ref, mass, sp, s.box, 1.0, 5, n_layers=2,
                            precision=mp.MP_FP32, n_parts=4, k_hops=2)
    # the sharded loop on one rank (the ranges are evaluated by one process)
    ops = LibraryOps(pot, sp, s.box, 2, mp.MP_FP32, 4)
    sysm = ShardedSystem(ops, 4)
    pos = torch.tensor(s.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    F, ledger = sysm.md(pos, vel, mass, 1.0, 5)
    torch.cuda.synchronize()
    assert np.abs(pos.cpu().numpy() - p_ref.cpu().numpy()).max() <= 1e-9
    assert np.abs(vel.cpu().numpy() - v_ref.cpu().numpy()).max() <= 1e-9
    assert np.allclose(np.array(ledger), led_ref, rtol=1e-10, atol=1e-9)
    assert np.array_equal(F.float().cpu().numpy(), f_ref.cpu().numpy()) or \
        np.abs(F.float().cpu().numpy() - f_ref.cpu().numpy()).max() <= 1e-6
    pot.close()
