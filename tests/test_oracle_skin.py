"""Oracle pins of the Verlet-skin reading: a neighbour list that also holds
pairs between r_c and r_c + skin gives the same energy and forces (the
envelope is zero from r_c on, the radial MLP is bias free, so R(r >= r_c) = 0
and those pairs add exact zeros), and partitions whose halos are built on
that list in units of r_c + skin stay exact."""
import numpy as np

import synth
from oracle import model as om
from oracle import neighbors as onb
from oracle import partition as op


def _system():
    s = synth.alloy_fcc(cells=(4, 4, 6), sigma=0.1, seed=6)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    return s, d, w


def test_pairs_beyond_cutoff_add_nothing():
    s, d, w = _system()
    e = onb.brute_force_edges(s.pos, s.box, d.r_cut)
    es = onb.brute_force_edges(s.pos, s.box, d.r_cut + 0.8)
    assert len(es[0]) > 1.3 * len(e[0])
    E0, Ei0, F0 = om.energy_forces(s.pos, s.species, s.box, e, w, d, 2)
    E1, Ei1, F1 = om.energy_forces(s.pos, s.species, s.box, es, w, d, 2)
    frms = np.sqrt((F0 ** 2).mean())
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.abs(Ei1 - Ei0).max() <= 1e-12 * np.abs(Ei0).max()
    assert np.abs(F1 - F0).max() <= 1e-12 * frms


def test_list_built_earlier_stays_exact_within_half_skin():
    """Atoms moved by less than skin / 2 since the list was built: every pair
    now within r_c is in the old r_c + skin list, so E and F are the exact
    ones; the partitioned evaluation with the old list and halos of
    K (r_c + skin) built on it is exact too."""
    s, d, w = _system()
    skin = 0.8
    x0 = onb.wrap(s.pos, s.box)                # the list's image shifts refer to these
    es = onb.brute_force_edges(x0, s.box, d.r_cut + skin)
    rng = np.random.default_rng(3)
    step = rng.normal(size=s.pos.shape)
    step *= (0.45 * skin / 2) / np.linalg.norm(step, axis=1).max()
    p1 = x0 + step                             # no wrap: the list's image shifts stay valid
    E_ref, _, F_ref = om.energy_forces(p1, s.species, s.box,
                                       onb.brute_force_edges(p1, s.box, d.r_cut), w, d, 2)
    # the old list, evaluated at the new positions (unwrapped, so its shifts apply)
    x = np.asarray(p1, dtype=np.float64)
    import torch
    pos_t = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    Ei = om.atom_energies(pos_t, s.species, s.box, *es, w, d, 2)
    (g,) = torch.autograd.grad(Ei.sum(), pos_t)
    frms = np.sqrt((F_ref ** 2).mean())
    assert abs(float(Ei.sum()) - E_ref) <= 1e-12 * abs(E_ref)
    assert np.abs(-g.numpy() - F_ref).max() <= 1e-12 * frms
    # partitions on the old list: geometric halo of K (r_c + skin) at the build positions
    parts, _ = op.plan(x0, s.box, es, 3, 2, d.r_cut + skin, mode="geom")
    E_p, F_p = 0.0, np.zeros_like(F_ref)
    for roots, ext in parts:
        gid = np.nonzero(ext)[0]
        le = op.sub_edges(es, ext)
        pt = torch.tensor(x[gid], dtype=torch.float64, requires_grad=True)
        Ep = (om.atom_energies(pt, s.species[gid], s.box, *le, w, d, 2)
              * torch.tensor(roots[gid].astype(np.float64))).sum()
        (gp,) = torch.autograd.grad(Ep, pt)
        E_p += float(Ep)
        F_p[gid] -= gp.numpy()
    assert abs(E_p - E_ref) <= 1e-11 * abs(E_ref)
    assert np.abs(F_p - F_ref).max() <= 1e-11 * frms
