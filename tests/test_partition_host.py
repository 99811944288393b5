"""The graph partitioner's host step (recursive greedy bisection of the
coarsest graph), called through the C ABI on the CPU: valid and balanced
parts, the unique zero-cut split of disconnected equal components, the
optimal split of a path, determinism, weights honoured."""
import numpy as np
import pytest

from oracle import partition as op


@pytest.fixture(scope="module")
def mp():
    from paper_2509_21694_gb300 import build
    build.build()
    from paper_2509_21694_gb300 import binding
    return binding


def _csr(n, pairs):
    """Symmetric CSR (row_ptr, col) and the directed edge list of undirected pairs."""
    recv = np.array([a for a, b in pairs] + [b for a, b in pairs], dtype=np.int64)
    send = np.array([b for a, b in pairs] + [a for a, b in pairs], dtype=np.int64)
    order = np.lexsort((send, recv))
    recv, send = recv[order], send[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, recv + 1, 1)
    return np.cumsum(row_ptr), send.astype(np.int32), (recv, send, np.zeros(len(recv), np.int8))


def _grid(nx, ny):
    pairs = []
    for y in range(ny):
        for x in range(nx):
            i = y * nx + x
            if x + 1 < nx:
                pairs.append((i, i + 1))
            if y + 1 < ny:
                pairs.append((i, i + nx))
    return pairs


def test_path_is_cut_once(mp):
    n = 10
    rp, col, e = _csr(n, [(i, i + 1) for i in range(n - 1)])
    part = mp.mp_partition_host_bisect(rp, col, 2, seed=3)
    assert sorted(op.part_weights(part, 2)) == [5, 5]
    assert op.edge_cut(part, e) == 1


def test_disconnected_equal_components_split_at_zero_cut(mp):
    # two 4 x 4 grids, no edge between them
    g = _grid(4, 4)
    rp, col, e = _csr(32, g + [(a + 16, b + 16) for a, b in g])
    part = mp.mp_partition_host_bisect(rp, col, 2, seed=1)
    assert op.edge_cut(part, e) == 0
    assert len(set(part[:16])) == 1 and len(set(part[16:])) == 1 and part[0] != part[16]


@pytest.mark.parametrize("k", [2, 3, 4, 7])
def test_grid_parts_valid_balanced_deterministic(mp, k):
    n = 12 * 12
    rp, col, e = _csr(n, _grid(12, 12))
    part = mp.mp_partition_host_bisect(rp, col, k, seed=5)
    assert part.min() == 0 and part.max() == k - 1
    w = op.part_weights(part, k)
    # each bisection targets its share of the weight to within one vertex
    assert w.max() - w.min() <= int(np.log2(k)) + 2, w
    assert np.array_equal(part, mp.mp_partition_host_bisect(rp, col, k, seed=5))
    # far below a random assignment's cut
    rnd = np.arange(n) % k
    assert op.edge_cut(part, e) < 0.5 * op.edge_cut(rnd, e)


def test_vertex_weights_are_honoured(mp):
    # a path whose first vertex weighs as much as the other nine together
    n = 10
    rp, col, e = _csr(n, [(i, i + 1) for i in range(n - 1)])
    vw = np.ones(n, np.int32)
    vw[0] = 9
    part = mp.mp_partition_host_bisect(rp, col, 2, seed=0, vertex_w=vw)
    heavy = part[0]
    assert np.all(part[1:] != heavy)


def test_one_part_and_bad_input(mp):
    rp, col, _ = _csr(4, [(0, 1), (1, 2), (2, 3)])
    assert np.all(mp.mp_partition_host_bisect(rp, col, 1) == 0)
    with pytest.raises(mp.MPError):
        mp.mp_partition_host_bisect(rp, np.array([0, 1, 2, 9, 1, 2], np.int32), 2)


def test_malformed_csr_and_negative_weights_are_refused(mp):
    """A row_ptr that decreases inside, a negative vertex or edge weight: the
    C entry point answers MP_ERR_ARG before it indexes anything."""
    rp, col, _ = _csr(4, [(0, 1), (1, 2), (2, 3)])
    bad = rp.copy()
    bad[2] = bad[3] + 1                  # row 1 would end past row 2's start
    with pytest.raises(mp.MPError):
        mp.mp_partition_host_bisect(bad, col, 2)
    with pytest.raises(mp.MPError):
        mp.mp_partition_host_bisect(rp, col, 2, vertex_w=np.array([1, -1, 1, 1]))
    with pytest.raises(mp.MPError):
        mp.mp_partition_host_bisect(rp, col, 2, edge_w=-np.ones(len(col), np.int32))
    with pytest.raises(ValueError):       # col shorter than row_ptr says
        mp.mp_partition_host_bisect(rp, col[:-1], 2)
