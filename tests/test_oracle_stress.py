"""Oracle stress sigma = (1/V) dE/d(strain) (autograd through the strained edge
vectors), pinned by mechanisms that do not use that derivative."""
import numpy as np
import pytest

import synth
from oracle import model as om
from oracle import neighbors as onb
from oracle import partition as op


def _system():
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.1, seed=4)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    return s, d, synth.make_weights(d, 1)


def test_normal_components_match_rescaled_systems():
    # Central differences of E over real rescalings of one axis (positions and
    # box, neighbour list rebuilt): V sigma_aa = dE/d(eps_aa).
    s, d, w = _system()
    _, _, _, sig = om.energy_forces_stress(s.pos, s.species, s.box,
                                           onb.edges(s.pos, s.box, d.r_cut), w, d, 2)
    vol = np.prod(s.box)
    h = 1e-5

    def e_of(ax, t):
        p, b = s.pos.copy(), s.box.copy()
        p[:, ax] *= 1 + t
        b[ax] *= 1 + t
        return om.energy(p, s.species, b, onb.edges(p, b, d.r_cut), w, d, 2)
    for ax in range(3):
        fd = (e_of(ax, h) - e_of(ax, -h)) / (2 * h) / vol
        assert abs(fd - sig[ax, ax]) <= 1e-6 * abs(sig[ax, ax])


def test_pair_term_closed_form():
    # With no message-passing layer E = sum e0 + 1/2 sum_e phi(r_e), and the
    # virial of a pair potential is sigma = 1/(2V) sum_e phi'(r) d d^T / r.
    s, d, w = _system()
    e = onb.edges(s.pos, s.box, d.r_cut)
    _, _, _, sig = om.energy_forces_stress(s.pos, s.species, s.box, e, w, d, 0)
    recv, send, code = e
    x = onb.wrap(s.pos, s.box)
    dv = x[send] - x[recv] + onb.decode_shift(code) * s.box
    r = np.sqrt((dv * dv).sum(1))
    xr = r / d.r_cut
    p = d.p_env
    u = 1 - (p + 1) * (p + 2) / 2 * xr ** p + p * (p + 2) * xr ** (p + 1) - p * (p + 1) / 2 * xr ** (p + 2)
    du = (-(p + 1) * (p + 2) / 2 * p * xr ** (p - 1) + p * (p + 2) * (p + 1) * xr ** p
          - p * (p + 1) / 2 * (p + 2) * xr ** (p + 1)) / d.r_cut
    s12 = (d.rep_sigma / r) ** 12
    dphi = d.rep_eps * (-12 * s12 / r * u + s12 * du)
    ref = (0.5 * dphi / r)[:, None, None] * dv[:, :, None] * dv[:, None, :]
    ref = ref.sum(0) / np.prod(s.box)
    assert np.abs(sig - ref).max() <= 1e-12 * np.abs(ref).max()


def test_stress_is_symmetric():
    # Rotation invariance of E makes dE/d(strain) symmetric.
    s, d, w = _system()
    _, _, _, sig = om.energy_forces_stress(s.pos, s.species, s.box,
                                           onb.edges(s.pos, s.box, d.r_cut), w, d, 2)
    assert np.abs(sig - sig.T).max() <= 1e-12 * np.abs(sig).max()
    assert np.abs(sig - np.diag(np.diag(sig))).max() > 1e-8   # shear present (disorder)


@pytest.mark.parametrize("mode", ["geom", "bfs"])
def test_partitioned_stress_sums_to_whole(mode):
    # Output integration: per-partition stress with root-only seeds sums to
    # the whole system's stress (linear in the seeds, like the forces).
    s = synth.alloy_fcc(cells=(4, 4, 10), sigma=0.1, seed=8)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    e = onb.edges(s.pos, s.box, d.r_cut)
    _, _, _, sig = om.energy_forces_stress(s.pos, s.species, s.box, e, w, d, 2)
    parts, _ = op.plan(s.pos, s.box, e, 4, 2, d.r_cut, mode)
    tot = np.zeros((3, 3))
    for roots, ext in parts:
        gid = np.nonzero(ext)[0]
        _, _, _, sp = om.energy_forces_stress(s.pos[gid], s.species[gid], s.box,
                                              op.sub_edges(e, ext), w, d, 2,
                                              seed_mask=roots[gid].astype(np.float64))
        tot += sp
    assert np.abs(tot - sig).max() <= 1e-11 * np.abs(sig).max()
