"""Pins of the oracle's layer diagnostics (MFS and linear CKA)."""
import math

import numpy as np

import synth
from oracle import diagnostics as od
from oracle import neighbors as onb


def test_cka_identities():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(200, 16))
    q, _ = np.linalg.qr(rng.normal(size=(16, 16)))
    assert abs(od.cka(x, x) - 1) < 1e-13
    assert abs(od.cka(x, 3.7 * x @ q) - 1) < 1e-12      # rotation and isotropic scale
    y = rng.normal(size=(200, 16))
    c = od.cka(x, y)
    assert 0 < c < 1 and abs(c - od.cka(y, x)) < 1e-14


def test_mfs_identities():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(50, 8))
    assert od.mfs(x, x) == 0.0
    assert od.mfs(x, x + 5.0) < 1e-13                   # a common shift is removed
    assert abs(od.mfs(x, 2 * x) - np.linalg.norm(od.centre(x)) / 50) < 1e-13


def test_two_node_example():
    # H1 = [[1, 0], [3, 0]], H2 = [[0, 1], [0, 5]]: centred [[-1, 0], [1, 0]] and
    # [[0, -2], [0, 2]].  MFS = ||[[1, -2], [-1, 2]]||_F / 2 = sqrt(10) / 2.
    # H1~^T H2~ = [[0, 4], [0, 0]] -> 16;  ||H1~^T H1~|| = 2, ||H2~^T H2~|| = 8.
    h1 = np.array([[1.0, 0.0], [3.0, 0.0]])
    h2 = np.array([[0.0, 1.0], [0.0, 5.0]])
    assert abs(od.mfs(h1, h2) - math.sqrt(10) / 2) < 1e-15
    assert abs(od.cka(h1, h2) - 16 / (2 * 8)) < 1e-15


def test_layer_stats_shapes_and_ranges():
    s = synth.alloy_fcc(cells=(4, 4, 4), sigma=0.1, seed=2)
    d = synth.model_alloy(n_layers_full=3)
    w = synth.make_weights(d, 1)
    m, c = od.layer_stats(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w, d, 3)
    assert m.shape == (3,) and c.shape == (3,)
    assert np.all(m > 0) and np.all((c > 0) & (c <= 1 + 1e-12))
