"""Oracle head-loss gradient pinned by finite differences and special cases."""
import numpy as np
import pytest

import synth
from oracle import head as oh
from oracle import model as om
from oracle import neighbors as nb


def _setup():
    s = synth.alloy_fcc(cells=(3, 3, 4), sigma=0.1, seed=4)
    d = synth.ModelDesc(n_species=2, F=16, lmax=2, n_layers_full=2, r_cut=4.0,
                        n_avg=synth.n_avg_for(4.0, 4 / 3.6 ** 3))
    d.head_hidden = 32
    w = synth.make_weights(d, 5)
    e = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    rng = np.random.default_rng(2)
    e_ref = 1.3 * len(s.pos)
    f_ref = rng.normal(0, 0.3, s.pos.shape)
    return s, d, w, e, e_ref, f_ref


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_head_gradient_matches_finite_differences(lam):
    s, d, w, e, e_ref, f_ref = _setup()
    L, g = oh.loss_and_grad(s.pos, s.species, s.box, e, w, d, 2, e_ref, f_ref, lam)
    theta = oh.pack(w)
    rng = np.random.default_rng(7)
    idx = list(rng.choice(theta.size, 10, replace=False)) + [theta.size - 1, theta.size - 40]
    h = 1e-5
    for q in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        Lp, _ = oh.loss_and_grad(s.pos, s.species, s.box, e, oh.unpack(tp, w), d, 2, e_ref, f_ref,
                                 lam, with_grad=False)
        Lm, _ = oh.loss_and_grad(s.pos, s.species, s.box, e, oh.unpack(tm, w), d, 2, e_ref, f_ref,
                                 lam, with_grad=False)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g).max()), (q, fd, g[q])


def test_zero_output_head_is_transparent():
    s, d, w, e, _, _ = _setup()
    w0 = dict(w)
    w0["head_W2"] = np.zeros_like(w["head_W2"])
    w0["head_b2"] = np.zeros_like(w["head_b2"])
    E1, _, F1 = om.energy_forces(s.pos, s.species, s.box, e, w0, d, 2, use_head=True)
    E0, _, F0 = om.energy_forces(s.pos, s.species, s.box, e, w0, d, 2, use_head=False)
    assert abs(E1 - E0) < 1e-12 * abs(E0) and np.allclose(F1, F0, atol=1e-14)
