"""GPU cell-list neighbour CSR against the FP64 oracle: bit-exact edge sets."""
import numpy as np
import pytest
import torch

import synth
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


def _gpu_edges(mp, pot, pos, box):
    g = mp.mp_build_neighbors(pot.ctx, torch.tensor(pos, device="cuda"), box)
    try:
        r, s, c = mp.mp_graph_export(g)
        n, ne = mp.mp_graph_info(g)
    finally:
        mp.mp_graph_free(g)
    r, s, c = r.cpu().numpy().astype(np.int64), s.cpu().numpy().astype(np.int64), c.cpu().numpy().astype(np.int64)
    assert len(r) == ne
    order = np.lexsort((c, s, r))
    return r[order], s[order], c[order]


def _pot(mp, r_cut):
    d = synth.model_c1()
    d.r_cut = r_cut
    return mp.Potential(d, synth.make_weights(d, 0))


@pytest.mark.parametrize("case", ["c1", "alloy4000", "liquid2000", "tiny_box", "unwrapped"])
def test_neighbors_bit_exact(mp, case):
    if case == "c1":
        s, rc = synth.cu_fcc_small(), 5.0
    elif case == "alloy4000":
        s, rc = synth.alloy_fcc(), 6.0
    elif case == "liquid2000":
        s, rc = synth.liquid3(n=2000), 6.0
    elif case == "tiny_box":      # 2 cells per axis: every cell is a candidate
        s, rc = synth.alloy_fcc(cells=(3, 4, 5), sigma=0.2), 5.0
    else:                         # coordinates far outside the box
        s, rc = synth.cu_fcc_small(), 5.0
        s.pos = s.pos + np.array([3, -2, 7]) * s.box + 1e-3
    pot = _pot(mp, rc)
    ref = onb.edges(s.pos, s.box, rc)
    got = _gpu_edges(mp, pot, s.pos, s.box)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_cutoff_boundary_exact(mp):
    # Pairs at exactly r_c (excluded, strict <) and one ulp inside (included).
    box = np.array([20.0, 20.0, 20.0])
    rc = 6.0
    inside = np.nextafter(6.0, 0.0)
    pos = np.array([[1.0, 1.0, 1.0], [7.0, 1.0, 1.0],            # exactly r_c
                    [1.0, 10.0, 1.0], [1.0 + inside, 10.0, 1.0],  # one ulp inside
                    [15.0, 15.0, 15.0], [15.0, 15.0, 15.0 - 6.0 * (1 + 1e-5)]])
    pot = _pot(mp, rc)
    ref = onb.edges(pos, box, rc)
    got = _gpu_edges(mp, pot, pos, box)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    pairs = set(zip(ref[0].tolist(), ref[1].tolist()))
    assert (2, 3) in pairs and (0, 1) not in pairs


def test_periodic_wrap_pair(mp):
    box = np.array([12.0, 13.0, 14.0])
    pos = np.array([[0.1, 6.0, 7.0], [11.9, 6.0, 7.0], [5.0, 0.05, 13.97]])
    pot = _pot(mp, 5.0)
    ref = onb.edges(pos, box, 5.0)
    got = _gpu_edges(mp, pot, pos, box)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_large_fcc_counts_and_symmetry(mp):
    # 64k displaced FCC atoms: rows of 78 +- noise; exact set vs oracle cell list.
    s = synth.cu_fcc_large(cells=(16, 16, 64), sigma=0.05, seed=3)
    pot = _pot(mp, 6.0)
    got = _gpu_edges(mp, pot, s.pos, s.box)
    ref = onb.cell_list_edges(s.pos, s.box, 6.0)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_error_codes(mp):
    pot = _pot(mp, 5.0)
    with pytest.raises(mp.MPError) as e:
        mp.mp_build_neighbors(pot.ctx, torch.zeros(4, 3, dtype=torch.float64, device="cuda") +
                              torch.arange(4, device="cuda")[:, None].double(), [9.0, 20.0, 20.0])
    assert e.value.code == -2
    pos = torch.tensor([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0 + 1e-4], [5.0, 5.0, 5.0]],
                       dtype=torch.float64, device="cuda")
    with pytest.raises(mp.MPError) as e:
        mp.mp_build_neighbors(pot.ctx, pos, [20.0, 20.0, 20.0])
    assert e.value.code == -3


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_position_is_refused(mp, bad):
    """A NaN or infinite coordinate is caught on the device (it would bin
    into cell 0 and silently lose its edges) and the call returns MP_ERR_ARG;
    the context stays usable."""
    pot = _pot(mp, 5.0)
    pos, box = synth.fcc((3, 3, 3), 3.615)
    p = torch.tensor(pos, device="cuda")
    p[7, 1] = bad
    with pytest.raises(mp.MPError) as e:
        mp.mp_build_neighbors(pot.ctx, p, box)
    assert e.value.code == -1
    ok = _gpu_edges(mp, pot, pos, box)
    ref = onb.edges(pos, box, 5.0)
    for a, b in zip(ref, ok):
        assert np.array_equal(a, b)


def test_dense_stencil_fallback_bit_exact(mp):
    # 2,500 atoms in a 12 A box with r_c = 5: 2 cells per axis, so every
    # stencil holds all atoms, more than a cell block stages in shared
    # memory; the warp-per-receiver search takes over and must agree too.
    pos, box = synth.rsa_liquid(2500, 2500 / 12.0 ** 3, 0.6, 17)
    pot = _pot(mp, 5.0)
    ref = onb.edges(pos, box, 5.0)
    got = _gpu_edges(mp, pot, pos, box)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
