"""Oracle neighbour sets against the definition and closed-form counts."""
import numpy as np
import pytest

import synth
from oracle import neighbors as nb


@pytest.mark.parametrize("cells,a,rc,expect", [((3, 3, 3), 3.615, 5.0, 42),
                                                ((4, 4, 4), 3.615, 6.0, 78),
                                                ((4, 4, 4), 3.6, 6.0, 78)])
def test_perfect_fcc_neighbour_count(cells, a, rc, expect):
    # FCC shells at a/sqrt2 * sqrt(n): 12, 6, 24, 12, 24, 8 atoms; r_c = 5
    # keeps n <= 3 (42), r_c = 6 keeps n <= 5 (78) for a = 3.6 and 3.615.
    pos, box = synth.fcc(cells, a)
    recv, send, code = nb.brute_force_edges(pos, box, rc)
    assert np.all(np.bincount(recv, minlength=pos.shape[0]) == expect)


def _check_edge_set_properties(pos, box, rc, e):
    recv, send, code = e
    x = nb.wrap(pos, box)
    n = nb.decode_shift(code)
    d = x[send] - x[recv] + n * box
    r = np.sqrt((d * d).sum(1))
    assert r.max() < rc
    assert np.all((recv != send) | np.any(n != 0, axis=1))
    # symmetric: (i <- j, n) exists iff (j <- i, -n) exists
    fwd = set(zip(recv.tolist(), send.tolist(), code.tolist()))
    back = set(zip(send.tolist(), recv.tolist(), nb.shift_code(-n).tolist()))
    assert fwd == back
    # rows sorted by (recv, send, code)
    key = recv * (10 ** 9) + send * 27 + code
    assert np.all(np.diff(key) > 0)


def test_brute_force_properties_small():
    s = synth.cu_fcc_small()
    e = nb.brute_force_edges(s.pos, s.box, 5.0)
    _check_edge_set_properties(s.pos, s.box, 5.0, e)


def test_brute_force_matches_naive_loop_tiny():
    # 20 random atoms in a 10.5 A box: a triple loop over all 27 images
    # (no minimum-image formula) gives the same directed edge set.
    rng = np.random.default_rng(0)
    box = np.array([10.5, 11.0, 12.0])
    pos = rng.random((20, 3)) * box
    rc = 5.0
    ref = set()
    for i in range(20):
        for j in range(20):
            for nx in (-1, 0, 1):
                for ny in (-1, 0, 1):
                    for nz in (-1, 0, 1):
                        if i == j and nx == ny == nz == 0:
                            continue
                        d = pos[j] + np.array([nx, ny, nz]) * box - pos[i]
                        if np.dot(d, d) < rc * rc:
                            ref.add((i, j, (nx + 1) * 9 + (ny + 1) * 3 + nz + 1))
    recv, send, code = nb.brute_force_edges(pos, box, rc)
    assert set(zip(recv.tolist(), send.tolist(), code.tolist())) == ref


@pytest.mark.parametrize("which", ["c1", "alloy", "liquid"])
def test_cell_list_bit_exact_vs_brute_force(which):
    if which == "c1":
        s, rc = synth.cu_fcc_small(), 5.0
    elif which == "alloy":
        s, rc = synth.alloy_fcc(cells=(5, 5, 6)), 6.0
    else:
        s, rc = synth.liquid3(n=1200), 6.0
    b = nb.brute_force_edges(s.pos, s.box, rc)
    c = nb.cell_list_edges(s.pos, s.box, rc)
    for u, v in zip(b, c):
        assert np.array_equal(u, v)
    _check_edge_set_properties(s.pos, s.box, rc, b)


def test_wrap_canonical():
    box = np.array([10.0, 10.0, 10.0])
    p = np.array([[-1e-18, 10.0, 25.0], [3.0, -7.5, 9.999999999999998]])
    w = nb.wrap(p, box)
    assert (w >= 0).all() and (w < box).all()
    assert w[0, 1] == 0.0 and w[0, 2] == 5.0 and w[1, 1] == 2.5


def test_box_too_small_rejected():
    with pytest.raises(ValueError):
        nb.brute_force_edges(np.zeros((2, 3)), np.array([9.0, 12.0, 12.0]), 5.0)
