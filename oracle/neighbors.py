"""Periodic neighbour sets, FP64 (oracle; test infrastructure only).

Definition (the geometry the method's message passing runs on; the paper's
atom graph connects atoms closer than the cutoff r_c, Introduction and
Methods "Graph Partitioning"):

* Orthorhombic box L = (Lx, Ly, Lz), periodic in all three directions, with
  min(L) >= 2 r_c so that at most one periodic image of an atom lies within
  r_c of another.
* Positions are first wrapped: x_w = x - L floor(x / L); a result equal to L
  (rounding of a tiny negative x) becomes x_w - L.
* Directed edge (i <- j) with integer image shift n in {-1,0,1}^3 exists iff
  i != j and r^2 < r_c^2 strictly, where, per axis,
      dx = fl(x_w[j] - x_w[i]),  n = -rint(dx / L),  d = fl(dx + n L),
      r^2 = fl(fl(fl(d_x d_x) + fl(d_y d_y)) + fl(d_z d_z))
  (IEEE binary64, round to nearest even, no fused multiply-add).
* Shift code = (n_x + 1) * 9 + (n_y + 1) * 3 + (n_z + 1); rows are sorted by
  (receiver, sender, shift code).

Parity pins: brute_force_edges is the definition itself; closed-form FCC
neighbour counts and the cell list's bit-exact equality with it are tested.
"""
from __future__ import annotations

import numpy as np


def wrap(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Canonical wrap of positions into [0, L) per axis."""
    w = pos - box * np.floor(pos / box)
    w = np.where(w >= box, w - box, w)
    return w


def _pair_geometry(xi: np.ndarray, xj: np.ndarray, box: np.ndarray):
    """Minimum-image displacement d = r_j - r_i + n*L and r^2, per the definition."""
    dx = xj - xi
    n = -np.rint(dx / box)
    d = dx + n * box
    r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]
    r2 = r2 + d[..., 2] * d[..., 2]
    return d, n.astype(np.int64), r2


def shift_code(n: np.ndarray) -> np.ndarray:
    return ((n[..., 0] + 1) * 9 + (n[..., 1] + 1) * 3 + (n[..., 2] + 1)).astype(np.int64)


def decode_shift(code: np.ndarray) -> np.ndarray:
    code = np.asarray(code, dtype=np.int64)
    return np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=-1)


def check_box(box: np.ndarray, r_cut: float) -> None:
    if np.min(box) < 2.0 * r_cut:
        raise ValueError("box narrower than 2 r_c: minimum image is not unique")


def brute_force_edges(pos: np.ndarray, box: np.ndarray, r_cut: float,
                      chunk: int = 512):
    """All directed edges by O(N^2) search.  Returns (recv, send, code) int64
    arrays sorted by (recv, send, code); positions are wrapped first."""
    check_box(box, r_cut)
    x = wrap(np.asarray(pos, dtype=np.float64), box)
    n = x.shape[0]
    rc2 = r_cut * r_cut
    R, S, C = [], [], []
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        _, sh, r2 = _pair_geometry(x[i0:i1, None, :], x[None, :, :], box)
        mask = r2 < rc2
        ii = np.arange(i0, i1)
        mask[ii - i0, ii] = False
        ri, sj = np.nonzero(mask)
        R.append(ri + i0)
        S.append(sj)
        C.append(shift_code(sh[ri, sj]))
    recv = np.concatenate(R)
    send = np.concatenate(S)
    code = np.concatenate(C)
    order = np.lexsort((code, send, recv))
    return recv[order], send[order], code[order]


def cell_list_edges(pos: np.ndarray, box: np.ndarray, r_cut: float):
    """Same edge set as brute_force_edges, found through a cell list.

    Cells are at least r_c + 1e-6 wide per axis, so every neighbour lies in
    the 27 surrounding cells (all cells of an axis with fewer than 3 cells).
    Each candidate pair is tested with the same FP64 formula as the
    definition.
    """
    check_box(box, r_cut)
    x = wrap(np.asarray(pos, dtype=np.float64), box)
    n = x.shape[0]
    nc = np.maximum(1, np.floor(box / (r_cut + 1e-6)).astype(np.int64))
    c = np.minimum((x / box * nc).astype(np.int64), nc - 1)
    cid = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    order = np.argsort(cid, kind="stable")
    ncell = int(np.prod(nc))
    start = np.searchsorted(cid[order], np.arange(ncell + 1))
    offs = []
    for ax in range(3):
        offs.append([-1, 0, 1] if nc[ax] >= 3 else None)
    rc2 = r_cut * r_cut
    R, S, C = [], [], []
    for cz in range(nc[2]):
        for cy in range(nc[1]):
            for cx in range(nc[0]):
                me = order[start[(cz * nc[1] + cy) * nc[0] + cx]:
                           start[(cz * nc[1] + cy) * nc[0] + cx + 1]]
                if me.size == 0:
                    continue
                cand = []
                zs = [(cz + o) % nc[2] for o in offs[2]] if offs[2] else range(nc[2])
                ys = [(cy + o) % nc[1] for o in offs[1]] if offs[1] else range(nc[1])
                xs = [(cx + o) % nc[0] for o in offs[0]] if offs[0] else range(nc[0])
                for zz in zs:
                    for yy in ys:
                        for xx in xs:
                            k = (zz * nc[1] + yy) * nc[0] + xx
                            cand.append(order[start[k]:start[k + 1]])
                cand = np.concatenate(cand)
                _, sh, r2 = _pair_geometry(x[me][:, None, :], x[cand][None, :, :], box)
                mask = (r2 < rc2) & (me[:, None] != cand[None, :])
                ri, sj = np.nonzero(mask)
                R.append(me[ri])
                S.append(cand[sj])
                C.append(shift_code(sh[ri, sj]))
    recv = np.concatenate(R) if R else np.zeros(0, np.int64)
    send = np.concatenate(S) if S else np.zeros(0, np.int64)
    code = np.concatenate(C) if C else np.zeros(0, np.int64)
    order = np.lexsort((code, send, recv))
    return recv[order], send[order], code[order]


def edges(pos, box, r_cut, brute_limit: int = 6000):
    """Edge set by the definition: brute force for small N, else the cell list."""
    if pos.shape[0] <= brute_limit:
        return brute_force_edges(pos, box, r_cut)
    return cell_list_edges(pos, box, r_cut)


def to_csr(recv: np.ndarray, n: int) -> np.ndarray:
    """Row pointer of a receiver-sorted edge list."""
    return np.searchsorted(recv, np.arange(n + 1)).astype(np.int64)
