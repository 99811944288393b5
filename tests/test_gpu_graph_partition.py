"""Graph-based Stage 1 on the GPU (Methods, "Graph Partitioning";
Supplementary S1).

* Plans from a caller-given assignment: sets bit-exact against the oracle's
  BFS extension; slab bins given as an assignment reproduce the slab plan.
* The multilevel partitioner: every atom in one of the n_parts parts, part
  sizes within the bound, the same output for the same seed, the reported
  cut equal to the oracle's count on the returned assignment; two
  disconnected components are separated at zero cut (the unique optimum);
  on particles on a support its halo factor is below the z grid's.
* Partitioned evaluation and MD with graph parts reproduce the
  unpartitioned results (exactness does not depend on the root sets).
"""
import math

import numpy as np
import pytest
import torch

import gates
import synth
from oracle import model as om
from oracle import neighbors as onb
from oracle import partition as op

pytestmark = pytest.mark.gpu


def _small_model(r_cut=5.0):
    d = synth.ModelDesc(n_species=2, F=64, lmax=1, n_layers_full=2, r_cut=r_cut,
                        n_avg=synth.n_avg_for(r_cut, 4 / 3.6 ** 3))
    return d, synth.make_weights(d, 31)


def _graph(mp, s, d, w):
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    return pot, pos, g


def _export_sets(mp, plan, p, n):
    gid, root = mp.mp_plan_export(plan, p)
    gid = gid.cpu().numpy()
    root = root.cpu().numpy().astype(bool)
    ext = np.zeros(n, bool)
    ext[gid] = True
    roots = np.zeros(n, bool)
    roots[gid[root]] = True
    return ext, roots, gid


def _bound(n, k, imbalance):
    return max(math.ceil(n / k), math.floor((1 + imbalance) * n / k))


def test_assign_plan_sets_match_oracle(mp):
    s = synth.supported_particles(seed=5)
    d, w = _small_model()
    n = len(s.pos)
    assign = (synth.seeded_permutation(n, 7, synth.STREAM_SPLIT) % 5).astype(np.int32)
    pot, pos, g = _graph(mp, s, d, w)
    plan, H = mp.mp_partition_assign(pot.ctx, g, torch.tensor(assign, device="cuda"), 5, 2)
    parts, Hr = op.assignment_plan(assign, onb.edges(s.pos, s.box, d.r_cut), 5, 2)
    try:
        for p, (roots, ext) in enumerate(parts):
            got_ext, got_roots, _ = _export_sets(mp, plan, p, n)
            assert np.array_equal(got_ext, ext)
            assert np.array_equal(got_roots, roots)
        assert abs(H - Hr) < 1e-12
    finally:
        mp.mp_plan_free(plan)
        mp.mp_graph_free(g)
        pot.close()


def test_assign_with_slab_bins_is_the_slab_plan(mp):
    s = synth.alloy_fcc(cells=(5, 5, 12), sigma=0.1, seed=8)
    d, w = _small_model(4.0)
    pot, pos, g = _graph(mp, s, d, w)
    bins = op.root_bins(s.pos, s.box, 4).astype(np.int32)
    pa, Ha = mp.mp_partition_assign(pot.ctx, g, torch.tensor(bins, device="cuda"), 4, 2)
    pb, Hb = mp.mp_partition(pot.ctx, g, 4, 2, mp.MP_HALO_BFS)
    try:
        assert Ha == Hb
        for p in range(4):
            ga, ra = mp.mp_plan_export(pa, p)
            gb, rb = mp.mp_plan_export(pb, p)
            # same classes, same placement order
            assert torch.equal(ga, gb) and torch.equal(ra, rb)
            assert mp.mp_plan_info(pa, p) == mp.mp_plan_info(pb, p)
    finally:
        mp.mp_plan_free(pa)
        mp.mp_plan_free(pb)
        mp.mp_graph_free(g)
        pot.close()


@pytest.mark.parametrize("bad", [-1, 4])
def test_assign_rejects_out_of_range(mp, bad):
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.05, seed=3)
    d, w = _small_model(4.0)
    pot, pos, g = _graph(mp, s, d, w)
    assign = np.zeros(len(s.pos), np.int32)
    assign[17] = bad
    try:
        with pytest.raises(mp.MPError) as ei:
            mp.mp_partition_assign(pot.ctx, g, torch.tensor(assign, device="cuda"), 4, 2)
        assert mp.ERRORS[ei.value.code] == "MP_ERR_ARG"
    finally:
        mp.mp_graph_free(g)
        pot.close()


@pytest.mark.parametrize("which", ["bulk", "particles"])
def test_graph_partition_valid_balanced_deterministic(mp, which):
    if which == "bulk":
        s = synth.alloy_fcc(cells=(10, 10, 10), sigma=0.08, seed=1)
    else:
        s = synth.supported_particles(cells_xy=(14, 14), slab_cells=3, radius=8.0, seed=6)
    d, w = _small_model()
    n = len(s.pos)
    e = onb.edges(s.pos, s.box, d.r_cut)
    pot, pos, g = _graph(mp, s, d, w)
    try:
        for k in (2, 3, 8):
            part, cut = mp.mp_graph_partition(pot.ctx, g, k, 0.03, seed=11)
            a = part.cpu().numpy()
            assert a.min() >= 0 and a.max() < k
            wts = op.part_weights(a, k)
            assert wts.min() > 0 and wts.max() <= _bound(n, k, 0.03), wts
            assert cut == op.edge_cut(a, e)
            part2, cut2 = mp.mp_graph_partition(pot.ctx, g, k, 0.03, seed=11)
            assert torch.equal(part, part2) and cut2 == cut
        part1, _ = mp.mp_graph_partition(pot.ctx, g, 1, 0.03)
        assert int(part1.abs().sum()) == 0
    finally:
        mp.mp_graph_free(g)
        pot.close()


def test_graph_partition_separates_components(mp):
    """Two FCC films 9.8 A apart (r_c = 5): the graph has two components of
    equal size, and the only zero-cut balanced bisection separates them."""
    a = 3.6
    film, _ = synth.fcc((6, 6, 3), a)
    gap = 8.0
    pos = np.concatenate([film, film + np.array([0, 0, 3 * a + gap])])
    box = np.array([6 * a, 6 * a, 2 * (3 * a + gap)])
    s = synth.System(synth.displace(pos, 0.05, 2), box, np.zeros(len(pos), np.int32),
                     np.full(len(pos), synth.MASS["Cu"]))
    d, w = _small_model()
    e = onb.edges(s.pos, s.box, d.r_cut)
    lower = np.arange(len(pos)) < len(film)
    assert not np.any(lower[e[0]] != lower[e[1]])    # no edge joins the films
    pot, _, g = _graph(mp, s, d, w)
    try:
        part, cut = mp.mp_graph_partition(pot.ctx, g, 2, 0.0, seed=3)
        a_ = part.cpu().numpy()
        assert cut == 0
        assert len(set(a_[lower])) == 1 and len(set(a_[~lower])) == 1
        assert a_[lower][0] != a_[~lower][0]
    finally:
        mp.mp_graph_free(g)
        pot.close()


def test_graph_partition_halo_below_z_grid_on_particles(mp):
    """Particles on a support, 8 parts, K = 2: the graph partition is
    balanced and its halo factor is below the z grid's (Supplementary S1:
    on heterogeneous geometry the graph partitioner's H is noticeably
    lower)."""
    s = synth.supported_particles(cells_xy=(24, 24), slab_cells=4, radius=12.0, seed=7)
    d, w = _small_model(6.0)
    n = len(s.pos)
    pot, pos, g = _graph(mp, s, d, w)
    try:
        part, cut = mp.mp_graph_partition(pot.ctx, g, 8, 0.03, seed=1)
        plan_g, H_graph = mp.mp_partition_assign(pot.ctx, g, part, 8, 2)
        plan_z, H_z = mp.mp_partition(pot.ctx, g, 8, 2, mp.MP_HALO_BFS)
        zbins = op.root_bins(s.pos, s.box, 8)
        wz = op.part_weights(zbins, 8)
        wg = op.part_weights(part.cpu().numpy(), 8)
        assert wg.max() <= _bound(n, 8, 0.03)
        assert wz.max() > 1.5 * n / 8            # the z grid is far from balanced
        assert H_graph < H_z, (H_graph, H_z)
        mp.mp_plan_free(plan_g)
        mp.mp_plan_free(plan_z)
    finally:
        mp.mp_graph_free(g)
        pot.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_partitioned_evaluation_with_graph_parts_is_exact(mp, precision):
    s = synth.supported_particles(seed=5)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    prec = mp.MP_FP32 if precision == "fp32" else mp.MP_BF16
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    part, _ = mp.mp_graph_partition(pot.ctx, g, 4, 0.03, seed=2)
    mp.mp_graph_free(g)
    E0, F0, e0 = pot.energy_forces(pos, sp, s.box, 2, precision=prec, per_atom=True)
    E1, F1, e1 = pot.energy_forces(pos, sp, s.box, 2, precision=prec, per_atom=True,
                                   n_parts=4, part=part)
    F0 = F0.cpu().numpy().astype(np.float64)
    F1 = F1.cpu().numpy().astype(np.float64)
    ok, gap = gates.output_gap(F1, F0)
    assert ok, gap
    f64 = [gates.fp64_forces(mp, pot, pos, sp, s.box, 2, prec),
           gates.fp64_forces(mp, pot, pos, sp, s.box, 2, prec, n_parts=4, part=part)]
    assert gates.fp64_gap(f64[1], f64[0]) <= gates.GATE, gates.fp64_gap(f64[1], f64[0])
    assert np.array_equal(e0.cpu().numpy(), e1.cpu().numpy())
    assert abs(E1.item() - E0.item()) <= 1e-9 * abs(E0.item())
    if precision == "fp32":
        Er, _, Fr = om.energy_forces(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut),
                                     w, d, 2)
        assert np.abs(F1 - Fr).max() <= 1e-5 * np.sqrt((Fr ** 2).mean())
    pot.close()


def test_md_with_graph_parts_matches_unpartitioned(mp):
    s = synth.supported_particles(seed=5)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    v0 = synth.maxwell(s.masses, 300.0, 3)
    out = []
    for use_parts in (False, True):
        pot = mp.Potential(d, w)
        pos = torch.tensor(s.pos, device="cuda")
        vel = torch.tensor(v0, device="cuda")
        frc = torch.zeros(len(s.pos), 3, dtype=torch.float32, device="cuda")
        part = None
        if use_parts:
            g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
            part, _ = mp.mp_graph_partition(pot.ctx, g, 4, 0.03, seed=2)
            mp.mp_graph_free(g)
        led = mp.mp_md_step(pot.ctx, pos, vel, frc, torch.tensor(s.masses, device="cuda"),
                            torch.tensor(s.species, device="cuda"), s.box, 1.0, 5, n_layers=2,
                            n_parts=4 if use_parts else 1, part=part)
        out.append((pos.cpu().numpy(), led))
        pot.close()
    dp = out[0][0] - out[1][0]
    dp -= s.box * np.round(dp / s.box)
    assert np.abs(dp).max() < 1e-7
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-7 * np.abs(out[0][1][:, 0]).max()


@pytest.mark.parametrize("which,k", [("particles", 2), ("liquid", 5), ("gas", 3), ("gas", 8)])
def test_graph_partition_exact_balance(mp, which, k):
    """With imbalance 0 every part holds at most ceil(N / k) atoms (the
    final exact balancing step), also for a sparse gas whose graph is
    mostly isolated atoms."""
    if which == "particles":
        s = synth.supported_particles(cells_xy=(14, 14), slab_cells=3, radius=8.0, seed=6)
    elif which == "liquid":
        s = synth.liquid3(n=2000, seed=2)
    else:
        pos, box = synth.rsa_liquid(3000, 0.002, 1.8, 5)
        s = synth.System(pos, box, np.zeros(3000, np.int32), np.ones(3000))
    d, w = _small_model()
    n = len(s.pos)
    e = onb.edges(s.pos, s.box, d.r_cut)
    pot, pos, g = _graph(mp, s, d, w)
    try:
        part, cut = mp.mp_graph_partition(pot.ctx, g, k, 0.0, seed=1)
        a = part.cpu().numpy()
        wts = op.part_weights(a, k)
        assert wts.max() <= math.ceil(n / k), wts
        assert cut == op.edge_cut(a, e)
    finally:
        mp.mp_graph_free(g)
        pot.close()
