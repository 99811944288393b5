"""Spatial-grid partitions with halos and the partitioned evaluation (oracle;
test infrastructure only).

Stage 1 (Methods, "Graph Partitioning"): the unit cell is divided into P
uniform bins along one axis (here z) and each atom becomes a root of the bin
of its scaled coordinate:  frac = x_w / L (x_w the canonical wrapped
coordinate), bin = min(floor(frac * P), P - 1).

Stage 2: each root set is extended so that every root keeps its full K-hop
neighbourhood.  Two extensions are provided:
* ``bfs_halo``: K breadth-first expansions over the global edge set, as the
  paper's Stage 2 does;
* ``geometric_halo``: every atom whose periodic z-distance to the slab
  [lo, hi) = [L p / P, L (p+1) / P) is below K r_c + 1e-6 Angstrom.  Every
  atom within K hops of a root is closer than K r_c to it, so this set
  contains the BFS set.
  distance of z outside the slab = min(d_lo, d_hi) with
      d_lo = lo - z        (z < lo)    or  lo + L - z   (z >= hi)
      d_hi = z - hi        (z >= hi)   or  z + L - hi   (z < lo)

Output integration (Methods, "Global Output Integration"): partition p is
evaluated on its extended set with the edges whose two ends both lie in it;
E = sum_p sum_{roots of p} E_i and F = sum_p -grad(sum_{roots of p} E_i), the
gradient scattered back to global atom ids (halo atoms receive force from
every partition that holds them).

Halo growth factor (Supplementary S1): H = (#halo atoms) / (#root atoms).

Stage 1 may also come from a graph partitioner (the paper uses METIS for
heterogeneous geometries): ``assignment_plan`` takes any per-atom
assignment and extends it by BFS; ``edge_cut`` and ``part_weights`` give the
two quantities such a partitioner trades off.

Parity pins: the partitioned E and F equal the unpartitioned ones (the
paper's exactness claim), BFS and geometric halos give equal root outputs,
the BFS set is contained in the geometric set, and roots cover every atom
exactly once.
"""
from __future__ import annotations

import numpy as np

from .neighbors import wrap
from .model import energy_forces


def root_bins(pos, box, n_parts: int, axis: int = 2) -> np.ndarray:
    x = wrap(np.asarray(pos, dtype=np.float64), box)[:, axis]
    frac = x / box[axis]
    return np.minimum(np.floor(frac * n_parts).astype(np.int64), n_parts - 1)


def geometric_halo(pos, box, n_parts: int, p: int, width: float, axis: int = 2):
    """Boolean mask of atoms within the slab or within ``width`` + 1e-6 of it."""
    L = box[axis]
    z = wrap(np.asarray(pos, dtype=np.float64), box)[:, axis]
    lo = (L * p) / n_parts
    hi = (L * (p + 1)) / n_parts
    roots = root_bins(pos, box, n_parts, axis) == p
    below = z < lo
    d_lo = np.where(below, lo - z, (lo + L) - z)
    d_hi = np.where(below, (z + L) - hi, z - hi)
    dist = np.minimum(d_lo, d_hi)
    return roots | (dist < width + 1e-6)


def bfs_halo(root_mask: np.ndarray, recv: np.ndarray, send: np.ndarray, k_hops: int):
    """Mask of atoms within k_hops edges of any root (roots included)."""
    mask = root_mask.copy()
    for _ in range(k_hops):
        frontier = mask[send]
        new = mask.copy()
        new[recv[frontier]] = True          # symmetric edge set
        mask = new
    return mask


def plan(pos, box, edges, n_parts: int, k_hops: int, r_cut: float, mode: str = "geom",
         axis: int = 2):
    """List of (roots_mask, extended_mask) per partition and the halo factor H."""
    recv, send, _ = edges
    bins = root_bins(pos, box, n_parts, axis)
    parts = []
    n_halo = 0
    for p in range(n_parts):
        roots = bins == p
        if mode == "geom":
            ext = geometric_halo(pos, box, n_parts, p, k_hops * r_cut, axis)
        elif mode == "bfs":
            ext = bfs_halo(roots, recv, send, k_hops)
        else:
            raise ValueError(mode)
        n_halo += int(ext.sum() - roots.sum())
        parts.append((roots, ext))
    H = n_halo / pos.shape[0]
    return parts, H


def assignment_plan(assign, edges, n_parts: int, k_hops: int):
    """Stage 1 by any partitioner, then Stage 2 by BFS: partition p has the
    roots {i : assign[i] = p} and their k_hops-hop neighbourhood (Methods,
    "Graph Partitioning"; the graph-based Stage 1 for heterogeneous systems).
    Returns the list of (roots_mask, extended_mask) and the halo factor H."""
    recv, send, _ = edges
    assign = np.asarray(assign)
    parts = []
    n_halo = 0
    for p in range(n_parts):
        roots = assign == p
        ext = bfs_halo(roots, recv, send, k_hops)
        n_halo += int(ext.sum() - roots.sum())
        parts.append((roots, ext))
    return parts, n_halo / assign.shape[0]


def edge_cut(assign, edges) -> int:
    """Undirected edges whose ends lie in different parts (each pair appears
    twice in the directed edge set)."""
    recv, send, _ = edges
    assign = np.asarray(assign)
    crossing = int((assign[recv] != assign[send]).sum())
    assert crossing % 2 == 0
    return crossing // 2


def part_weights(assign, n_parts: int) -> np.ndarray:
    """Atoms per part."""
    return np.bincount(np.asarray(assign), minlength=n_parts)


def sub_edges(edges, ext_mask):
    """Edges with both ends in the extended set, re-indexed to local ids
    (local order = increasing global id)."""
    recv, send, code = edges
    keep = ext_mask[recv] & ext_mask[send]
    g2l = -np.ones(ext_mask.shape[0], dtype=np.int64)
    g2l[np.nonzero(ext_mask)[0]] = np.arange(int(ext_mask.sum()))
    return g2l[recv[keep]], g2l[send[keep]], code[keep]


def partitioned_energy_forces(pos, species, box, edges, w, desc, n_layers, parts,
                              use_head=False):
    """E, per-atom root energies and F assembled from independent partitions."""
    n = pos.shape[0]
    E = 0.0
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    for roots, ext in parts:
        gid = np.nonzero(ext)[0]
        le = sub_edges(edges, ext)
        Ep, Eip, Fp = energy_forces(pos[gid], species[gid], box, le, w, desc, n_layers,
                                    seed_mask=roots[gid].astype(np.float64),
                                    use_head=use_head)
        E += Ep
        r = roots[gid]
        Ei[gid[r]] = Eip[r]
        F[gid] += Fp
    return E, Ei, F


def local_energy_force(pos, species, box, w, desc, n_layers, k, use_head=False):
    """E_k and F_k of one atom of an arbitrarily large periodic system, exact.

    Only atoms within K hops of k have energies that depend on r_k, and each
    hop is shorter than r_c, so roots = {i : |r_i - r_k| < K r_c} (minimum
    image).  Their energies are exact on the extended set
    {j : |r_j - r_k| < 2 K r_c} with the edges among it (the partition
    argument above applied to one spherical root set), and
    F_k = -d(sum_roots E_i)/d r_k.
    """
    from .neighbors import brute_force_edges
    x = wrap(np.asarray(pos, dtype=np.float64), box)
    d = x - x[k]
    d -= box * np.round(d / box)
    r = np.sqrt((d * d).sum(1))
    K = n_layers
    roots = r < K * desc.r_cut
    ext = r < 2 * K * desc.r_cut + 1e-6
    gid = np.nonzero(ext)[0]
    sub = x[gid]
    e = brute_force_edges(sub, box, desc.r_cut)
    _, Ei, F = energy_forces(sub, species[gid], box, e, w, desc, n_layers,
                             seed_mask=roots[gid].astype(np.float64), use_head=use_head)
    kl = int(np.searchsorted(gid, k))
    return float(Ei[kl]), F[kl]
