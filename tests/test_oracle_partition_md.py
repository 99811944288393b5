"""Oracle partition emulation (exactness claim) and velocity-Verlet pins."""
import math

import numpy as np
import pytest

import synth
from oracle import md as omd
from oracle import model as om
from oracle import neighbors as nb
from oracle import partition as op


def _small_alloy_model(n_layers):
    d = synth.ModelDesc(n_species=2, F=16, lmax=2, n_layers_full=n_layers, r_cut=4.0,
                        n_avg=synth.n_avg_for(4.0, 4 / 3.6 ** 3), rep_eps=0.3)
    return d, synth.make_weights(d, 21)


@pytest.mark.parametrize("K,P,mode", [(1, 4, "geom"), (2, 4, "geom"), (2, 4, "bfs"),
                                      (2, 3, "bfs"), (3, 5, "geom")])
def test_partitioned_equals_unpartitioned(K, P, mode):
    s = synth.alloy_fcc(cells=(5, 5, 10), sigma=0.1, seed=8)
    d, w = _small_alloy_model(3)
    e = nb.edges(s.pos, s.box, d.r_cut)
    E, Ei, F = om.energy_forces(s.pos, s.species, s.box, e, w, d, K)
    parts, H = op.plan(s.pos, s.box, e, P, K, d.r_cut, mode)
    # roots cover every atom exactly once
    cover = sum(r.astype(int) for r, _ in parts)
    assert np.all(cover == 1)
    Ep, Eip, Fp = op.partitioned_energy_forces(s.pos, s.species, s.box, e, w, d, K, parts)
    frms = np.sqrt((F ** 2).mean())
    assert abs(Ep - E) < 1e-12 * abs(E)
    assert np.allclose(Eip, Ei, atol=1e-12)
    assert np.abs(Fp - F).max() < 1e-11 * frms
    assert H > 0


def test_bfs_halo_inside_geometric_halo():
    s = synth.alloy_fcc(cells=(5, 5, 10), sigma=0.1, seed=8)
    e = nb.edges(s.pos, s.box, 4.0)
    for K in (1, 2):
        pg, Hg = op.plan(s.pos, s.box, e, 4, K, 4.0, "geom")
        pb, Hb = op.plan(s.pos, s.box, e, 4, K, 4.0, "bfs")
        for (rg, xg), (rb, xb) in zip(pg, pb):
            assert np.array_equal(rg, rb)
            assert np.all(xg[xb])
        assert Hb <= Hg


def test_truncated_halo_breaks_exactness():
    # A planted mistake: one hop too few must change the root forces, so the
    # equality test above can fail.
    s = synth.alloy_fcc(cells=(5, 5, 10), sigma=0.1, seed=8)
    d, w = _small_alloy_model(2)
    e = nb.edges(s.pos, s.box, d.r_cut)
    _, _, F = om.energy_forces(s.pos, s.species, s.box, e, w, d, 2)
    parts, _ = op.plan(s.pos, s.box, e, 4, 1, d.r_cut, "bfs")
    _, _, Fp = op.partitioned_energy_forces(s.pos, s.species, s.box, e, w, d, 2, parts)
    assert np.abs(Fp - F).max() > 1e-6 * np.sqrt((F ** 2).mean())


def test_root_bins_floor_rule():
    box = np.array([10.0, 10.0, 8.0])
    pos = np.array([[0, 0, 0.0], [0, 0, 1.999999], [0, 0, 2.0], [0, 0, 7.9999999], [0, 0, -1e-9]])
    assert op.root_bins(pos, box, 4).tolist() == [0, 0, 1, 3, 3]


def test_verlet_harmonic_closed_form():
    # 1-D oscillator F = -k x.  Velocity Verlet advances (x, v) by an exact
    # linear map whose rotation angle theta obeys cos(theta) = 1 - (w dt)^2/2,
    # so x_n = x0 cos(n theta) + v0 dt sin(n theta) / sin(theta) (from the
    # map's eigen-decomposition).
    m = np.array([2.0])
    k = 3.0 * synth.KAPPA ** -1
    w2 = k * synth.KAPPA / m[0]
    dt = 0.3
    x0, v0 = 0.7, 0.2

    def force(p):
        return 0.5 * k * float(p[0, 0] ** 2), -k * p * np.array([[1.0, 0, 0]])

    pos = np.array([[x0, 0.0, 0.0]])
    vel = np.array([[v0, 0.0, 0.0]])
    n = 40
    p, v, _, led = omd.verlet(pos, vel, m, None, force, dt, n)
    theta = math.acos(1 - w2 * dt * dt / 2)
    xn = x0 * math.cos(n * theta) + v0 * dt * math.sin(n * theta) / math.sin(theta)
    assert abs(p[0, 0] - xn) < 1e-12


def test_verlet_energy_error_scales_dt2():
    m = np.array([1.0])
    k = 1.0 / synth.KAPPA

    def force(p):
        return 0.5 * k * float(p[0, 0] ** 2), -k * p * np.array([[1.0, 0, 0]])

    errs = []
    for dt in (0.2, 0.1):
        n = int(round(6.0 / dt))
        _, _, _, led = omd.verlet(np.array([[1.0, 0, 0]]), np.zeros((1, 3)), m, None,
                                  force, dt, n)
        errs.append(np.abs(led[:, 2] - 0.5 * k).max())
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_drift_slope_units():
    led = np.zeros((10, 3))
    led[:, 2] = 5.0 + 2e-3 * np.arange(1, 11)     # +2 meV per step total
    # 100 atoms, dt = 1 fs: 2e-3 eV / 100 atoms per fs = 0.02 meV/atom/fs = 20 meV/atom/ps
    assert abs(omd.drift_mev_per_atom_ps(led, 100, 1.0) - 20.0) < 1e-9


def test_local_cluster_force_equals_full_evaluation():
    # One atom's E and F from its local cluster equal the whole-system result.
    s = synth.alloy_fcc(cells=(8, 8, 8), sigma=0.1, seed=2)
    d = synth.ModelDesc(n_species=2, F=16, lmax=2, n_layers_full=2, r_cut=3.5, n_avg=20.0)
    w = synth.make_weights(d, 3)
    E, Ei, F = om.energy_forces(s.pos, s.species, s.box, nb.edges(s.pos, s.box, d.r_cut), w, d, 2)
    for k in (5, 777, 2047):
        Ek, Fk = op.local_energy_force(s.pos, s.species, s.box, w, d, 2, k)
        assert abs(Ek - Ei[k]) <= 1e-12 * abs(Ei[k])
        assert np.abs(Fk - F[k]).max() <= 1e-12 * max(1.0, np.abs(F[k]).max())


def test_assignment_plan_with_slab_bins_is_the_bfs_plan():
    """Stage 1 given as an assignment reproduces the spatial-grid BFS plan."""
    s = synth.alloy_fcc(cells=(5, 5, 10), sigma=0.1, seed=8)
    e = nb.edges(s.pos, s.box, 4.0)
    bins = op.root_bins(s.pos, s.box, 4)
    pa, Ha = op.assignment_plan(bins, e, 4, 2)
    pb, Hb = op.plan(s.pos, s.box, e, 4, 2, 4.0, "bfs")
    assert Ha == Hb
    for (ra, xa), (rb, xb) in zip(pa, pb):
        assert np.array_equal(ra, rb) and np.array_equal(xa, xb)


def test_partitioned_equals_unpartitioned_for_any_assignment():
    """Exactness does not depend on the shape of the root sets: a random
    (fragmented) assignment and a supported-particle system both reproduce
    the unpartitioned energy and forces."""
    d, w = _small_alloy_model(2)
    for s, assign in [
        (synth.alloy_fcc(cells=(5, 5, 5), sigma=0.1, seed=9),
         synth.seeded_permutation(500, 3, synth.STREAM_SPLIT) % 3),
        (synth.supported_particles(cells_xy=(6, 6), slab_cells=2, radius=4.5, grid=(1, 1),
                                   seed=4), None),
    ]:
        e = nb.edges(s.pos, s.box, d.r_cut)
        if assign is None:   # quadrants of the xy plane
            x = nb.wrap(s.pos, s.box)
            assign = (2 * (x[:, 0] >= s.box[0] / 2) + (x[:, 1] >= s.box[1] / 2)).astype(int)
        P = int(assign.max()) + 1
        E, Ei, F = om.energy_forces(s.pos, s.species, s.box, e, w, d, 2)
        parts, H = op.assignment_plan(assign, e, P, 2)
        Ep, Eip, Fp = op.partitioned_energy_forces(s.pos, s.species, s.box, e, w, d, 2, parts)
        frms = np.sqrt((F ** 2).mean())
        assert abs(Ep - E) < 1e-12 * abs(E)
        assert np.allclose(Eip, Ei, atol=1e-12)
        assert np.abs(Fp - F).max() < 1e-11 * frms
        # one hop too few breaks it (the halo depth is what exactness needs)
        short, _ = op.assignment_plan(assign, e, P, 1)
        _, _, Fs = op.partitioned_energy_forces(s.pos, s.species, s.box, e, w, d, 2, short)
        assert np.abs(Fs - F).max() > 1e-6 * frms


def test_edge_cut_and_weights_by_hand():
    """A 4-cycle 0-1-2-3-0 split {0,1} | {2,3} cuts edges 1-2 and 3-0."""
    und = [(0, 1), (1, 2), (2, 3), (3, 0)]
    recv = np.array([a for a, b in und] + [b for a, b in und])
    send = np.array([b for a, b in und] + [a for a, b in und])
    edges = (recv, send, np.zeros(8, np.int8))
    assert op.edge_cut([0, 0, 1, 1], edges) == 2
    assert op.edge_cut([0, 1, 0, 1], edges) == 4
    assert op.edge_cut([0, 0, 0, 0], edges) == 0
    assert list(op.part_weights([0, 0, 1, 1], 3)) == [2, 2, 0]
    # BFS halo of root {0} with one hop: its two neighbours; H = 2 / 4 per part sum
    parts, H = op.assignment_plan(np.array([0, 1, 1, 1]), edges, 2, 1)
    assert list(np.nonzero(parts[0][1])[0]) == [0, 1, 3]
    assert list(np.nonzero(parts[1][1])[0]) == [0, 1, 2, 3]
    assert H == (2 + 1) / 4


def test_per_layer_receiver_edges_suffice():
    """Inside one partition, layer t only needs the edges whose receiver lies
    within K-1-t hops of a root: restricting every layer to those edges
    leaves the root energies and all forces unchanged.  In particular an
    edge whose two ends are both exactly K-t hops out is used at no layer
    >= t, in neither direction, so it contributes nothing to the adjoint of
    layer t (the edges the GPU adjoint skips); and a receiver set one hop
    smaller changes the result."""
    s = synth.alloy_fcc(cells=(5, 5, 10), sigma=0.1, seed=8)
    d, w = _small_alloy_model(3)
    e = nb.edges(s.pos, s.box, d.r_cut)
    recv, send, code = e
    K = 2
    roots = op.root_bins(s.pos, s.box, 4) == 1
    level = np.full(len(s.pos), K + 1)
    level[roots] = 0
    for h in range(1, K + 1):      # BFS levels over the symmetric edge set
        reach = np.zeros(len(s.pos), bool)
        reach[recv[level[send] < h]] = True
        level[(level > K) & reach] = h
    ext = level <= K
    gid = np.nonzero(ext)[0]
    lr, ls, lc = op.sub_edges(e, ext)
    lev = level[gid]
    seed = roots[gid].astype(np.float64)
    args = (s.pos[gid], s.species[gid], s.box, (lr, ls, lc), w, d, K)
    E0, Ei0, F0 = om.energy_forces(*args, seed_mask=seed)
    masks = [lev[lr] <= K - 1 - t for t in range(K)]
    E1, Ei1, F1 = om.energy_forces(*args, seed_mask=seed, layer_masks=masks)
    frms = np.sqrt((F0 ** 2).mean())
    assert abs(E1 - E0) < 1e-12 * abs(E0)
    assert np.abs(F1 - F0).max() < 1e-11 * frms
    # the edges dropped at layer t include every edge between two atoms of
    # level K - t, in both directions
    for t in range(K):
        outer = (lev[lr] == K - t) & (lev[ls] == K - t)
        assert outer.any() and not np.any(masks[t] & outer)
    # one level too few at the first layer is not enough
    short = [lev[lr] <= K - 2 - t for t in range(K)]
    _, _, F2 = om.energy_forces(*args, seed_mask=seed, layer_masks=short)
    assert np.abs(F2 - F0).max() > 1e-6 * frms
