"""Pins of the oracle and the shared generators against the cited fixtures
in tests/golden/ (closed forms and published values, not oracle output)."""
import os
from fractions import Fraction
from itertools import product

import numpy as np
import torch

import synth
from oracle import model as om
from oracle import neighbors as nb

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_fcc_shells_by_enumeration_and_oracle_counts():
    shells = [(int(s), float(r2), int(c)) for s, r2, c in _rows("fcc_shells.txt")]
    # the fixture itself: integer vectors with an even sum, |v|^2 = 2 s
    for s, r2, c in shells:
        assert r2 == s / 2
        n = sum(1 for v in product(range(-4, 5), repeat=3)
                if sum(v) % 2 == 0 and v[0] ** 2 + v[1] ** 2 + v[2] ** 2 == 2 * s)
        assert n == c
    # the oracle's neighbour list on perfect lattices
    for a, rc, cells in ((3.615, 5.0, (4, 4, 4)), (3.6, 6.0, (4, 4, 4))):
        pos, box = synth.fcc(cells, a)
        recv, _, _ = nb.edges(pos, box, rc)
        expect = sum(c for s, r2, c in shells if r2 * a * a < rc * rc)
        assert np.all(np.bincount(recv, minlength=len(pos)) == expect)
    assert sum(c for s, r2, c in shells[:3]) == 42 and sum(c for s, r2, c in shells[:5]) == 78


def test_splitmix64_published_outputs():
    want = [int(v, 16) for (v,) in _rows("splitmix64_seed0.txt")]
    gamma = 0x9E3779B97F4A7C15
    keys = np.array([0, gamma, (2 * gamma) % 2 ** 64], dtype=np.uint64)
    got = [int(x) for x in synth.splitmix64(keys)]
    assert got == want


def test_envelope_exact_values():
    for xn, xd, un, ud in _rows("envelope_p6.txt"):
        x = Fraction(int(xn), int(xd))
        u = Fraction(int(un), int(ud))
        # the fixture against the polynomial in exact arithmetic
        if x < 1:
            assert 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8 == u
        # the oracle in FP64 (these values are exact binary fractions)
        got = float(om.envelope(torch.tensor([float(x)], dtype=torch.float64), 6)[0])
        assert got == float(u)
