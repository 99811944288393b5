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
