"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds no arithmetic of the interatomic-potential method itself:
it only draws random numbers and lays out structures, velocities and weight
tensors.  Both sides receive what it returns as plain numpy arrays, so the
oracle and the CUDA library never share code, only inputs.

Random numbers come from one counter-based generator: the splitmix64 output
function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to the key ``seed ^ (stream << 40) ^ idx``.
A draw therefore never depends on the order in which draws are made.

Units: Angstrom, eV, amu, fs, K.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream keys for non-weight draws (weights use tensor ids below 0x100).
STREAM_DISPLACE = 0x101
STREAM_SPECIES = 0x102
STREAM_VELOCITY = 0x103
STREAM_LIQUID = 0x104
STREAM_SPLIT = 0x105
STREAM_LANGEVIN = 0x106   # thermostat noise, index (step * N + atom) * 3 + axis

KB_EV = 8.617333262e-5            # Boltzmann constant, eV/K
KAPPA = 9.648533212e-3            # 1 eV/(Angstrom*amu) in Angstrom/fs^2
MASS = {"Cu": 63.546, "Ni": 58.6934, "Al": 26.9815}


def splitmix64(state) -> np.ndarray:
    """First splitmix64 output for generator state ``state`` (uint64 array).

    The state is advanced by the golden gamma and then mixed by two
    xor-shift-multiply rounds and a final xor-shift (the published mixer).
    """
    with np.errstate(over="ignore"):
        z = np.asarray(state, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """U[0,1) draws with 53 random bits, counter-based on (seed, stream, idx)."""
    idx = np.asarray(idx, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40)) ^ idx
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on draws 2k (radius) and 2k+1 (angle)."""
    return normal_at(seed, stream, np.arange(n, dtype=np.uint64))


def normal_at(seed: int, stream: int, k) -> np.ndarray:
    """Standard normals number k (any counters) of the construction above."""
    k = np.asarray(k, dtype=np.uint64)
    u1 = 1.0 - uniform(seed, stream, np.uint64(2) * k)          # (0, 1]: log is finite
    u2 = uniform(seed, stream, np.uint64(2) * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# Model hyper-parameters and weights
# ----------------------------------------------------------------------------

@dataclass
class ModelDesc:
    """Hyper-parameters of the synthetic equivariant message-passing potential.

    n_species  S      number of chemical species
    F                 channels per (l, m) feature block
    lmax              highest spherical-harmonic degree (1 or 2)
    n_layers_full     L_full, depth of the unpruned network (weights exist for
                      all of them; a pruned run uses the first K)
    H                 hidden width of the radial MLP
    n_basis           number of Bessel radial functions
    p_env             polynomial cutoff envelope exponent
    r_cut             cutoff radius, Angstrom
    n_avg             fixed message normaliser (never data dependent)
    rep_eps, rep_sigma  optional pair repulsion eps*(sigma/r)^12*u(r/rc);
                      rep_eps = 0 disables it
    head_hidden       hidden width of the per-atom correction head
    """
    n_species: int = 1
    F: int = 64
    lmax: int = 1
    n_layers_full: int = 2
    H: int = 64
    n_basis: int = 8
    p_env: int = 6
    r_cut: float = 5.0
    n_avg: float = 44.0
    rep_eps: float = 0.0
    rep_sigma: float = 1.5
    head_hidden: int = 32

    @property
    def n_radial(self) -> int:
        """Radial MLP outputs: R0 plus (R_la, R_lb) for l = 1..lmax."""
        return self.F * (1 + 2 * self.lmax)

    @property
    def n_lm(self) -> int:
        return (self.lmax + 1) ** 2

    def to_dict(self):
        return asdict(self)


def n_avg_for(r_cut: float, density: float) -> float:
    """Nominal neighbour count (4 pi / 3) r_c^3 rho for a nominal density."""
    return 4.0 / 3.0 * math.pi * r_cut ** 3 * density


# Tensor ids of the counter-based weight generator.
TID_EMB, TID_E0, TID_WOUT = 1, 2, 3
TID_HEAD_W1, TID_HEAD_B1, TID_HEAD_W2, TID_HEAD_B2 = 8, 9, 10, 11
LAYER_TID_BASE, LAYER_TID_STRIDE = 16, 16
LAYER_TENSORS = ("W1", "W2", "W3", "W0", "U1", "U2", "b", "V1", "V2")

# Gains chosen so that the synthetic network is clearly nonlinear and the
# forces of the bulk configurations are O(0.1 - 1) eV/Angstrom.
DEFAULT_GAINS = {
    "emb": 1.0, "e0": 0.0, "w_out": 2.0,
    "W1": 3.0, "W2": 3.0, "W3": 3.0, "W0": 1.0, "U1": 1.0 / 3.0,
    "U2": 1.0 / 5.0, "b": 0.1, "V1": 1.0, "V2": 1.0,
    "head_W1": 1.0, "head_b1": 0.1, "head_W2": 1.0, "head_b2": 0.0,
}


def _tensor(seed, tid, shape, fan_in, gain):
    n = int(np.prod(shape))
    u = uniform(seed, tid, np.arange(n, dtype=np.uint64))
    return (gain * math.sqrt(3.0) * (2.0 * u - 1.0) / math.sqrt(fan_in)).reshape(shape)


def make_weights(desc: ModelDesc, seed: int, gains: dict | None = None) -> dict:
    """All weight tensors of ``desc`` as float64 numpy arrays.

    w[tid, idx] = gain * sqrt(3) * (2u - 1) / sqrt(fan_in), u = uniform(seed,
    tid, idx), idx the row-major flat index.  Layer tensors carry a leading
    axis of length n_layers_full.  Shapes (out, in) act as out = W @ in.
    """
    g = dict(DEFAULT_GAINS)
    if gains:
        g.update(gains)
    S, F, H, NB, P = desc.n_species, desc.F, desc.H, desc.n_basis, desc.n_radial
    w = {
        "emb": _tensor(seed, TID_EMB, (S, F), 1, g["emb"]),
        "e0": _tensor(seed, TID_E0, (S,), 1, g["e0"]),
        "w_out": _tensor(seed, TID_WOUT, (F,), F, g["w_out"]),
        "head_W1": _tensor(seed, TID_HEAD_W1, (desc.head_hidden, F), F, g["head_W1"]),
        "head_b1": _tensor(seed, TID_HEAD_B1, (desc.head_hidden,), 1, g["head_b1"]),
        "head_W2": _tensor(seed, TID_HEAD_W2, (desc.head_hidden,), desc.head_hidden, g["head_W2"]),
        "head_b2": _tensor(seed, TID_HEAD_B2, (1,), 1, g["head_b2"]),
    }
    shapes = {"W1": ((H, NB), NB), "W2": ((H, H), H), "W3": ((P, H), H),
              "W0": ((F, F), F), "U1": ((F, F), F), "U2": ((F, F), F),
              "b": ((F,), 1), "V1": ((F, F), F), "V2": ((F, F), F)}
    for k, name in enumerate(LAYER_TENSORS):
        shp, fan = shapes[name]
        w[name] = np.stack([
            _tensor(seed, LAYER_TID_BASE + LAYER_TID_STRIDE * t + k, shp, fan, g[name])
            for t in range(desc.n_layers_full)])
    if desc.lmax < 2:
        w["U2"] = w["U2"][:, :0, :0]
        w["V2"] = w["V2"][:, :0, :0]
    return w


# ----------------------------------------------------------------------------
# Structures
# ----------------------------------------------------------------------------

def fcc(cells, a: float) -> tuple[np.ndarray, np.ndarray]:
    """Perfect FCC lattice of cells = (nx, ny, nz) cubic cells of edge a.

    Atoms are listed cell by cell (x fastest, then y, then z) with the four
    basis sites (0,0,0), (0,.5,.5), (.5,0,.5), (.5,.5,0) inside each cell.
    Returns (positions [N,3], box [3]).
    """
    nx, ny, nz = cells
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origin = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (origin[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return pos, box


def displace(pos: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Add independent N(0, sigma^2) displacements to every coordinate."""
    return pos + sigma * normal(seed, STREAM_DISPLACE, pos.size).reshape(pos.shape)


def seeded_permutation(n: int, seed: int, stream: int) -> np.ndarray:
    """Permutation of range(n): indices sorted by their (seed, stream) draws."""
    keys = splitmix64(np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40))
                      ^ np.arange(n, dtype=np.uint64))
    return np.argsort(keys, kind="stable")


def assign_species(n: int, fractions, seed: int) -> np.ndarray:
    """Species index per atom: exact counts round(f*n) (last takes the rest),
    placed by a seeded shuffle."""
    counts = [int(round(f * n)) for f in fractions[:-1]]
    counts.append(n - sum(counts))
    labels = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in enumerate(counts)])
    out = np.empty(n, dtype=np.int32)
    out[seeded_permutation(n, seed, STREAM_SPECIES)] = labels
    return out


def rsa_liquid(n: int, density: float, d_min: float, seed: int,
               max_tries: int = 10_000) -> tuple[np.ndarray, np.ndarray]:
    """Random sequential addition of n atoms in a periodic cube of volume n/density.

    Candidate k (k = 0, 1, 2, ...) uses draws 3k..3k+2 of the liquid stream; it
    is accepted if its minimum-image distance to every accepted atom is at
    least d_min.  Raises RuntimeError after max_tries rejections in a row.
    """
    L = (n / density) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    nc = max(1, int(L // d_min))
    cw = L / nc
    cells: dict = {}
    pos = np.empty((n, 3))
    placed = 0
    cand = 0
    fails = 0
    batch = 4096
    while placed < n:
        k = np.arange(cand, cand + batch, dtype=np.uint64)
        xyz = np.stack([uniform(seed, STREAM_LIQUID, 3 * k + c) for c in range(3)], 1) * L
        cand += batch
        for p in xyz:
            c = tuple((p // cw).astype(int) % nc)
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        lst = cells.get(((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc))
                        if not lst:
                            continue
                        q = pos[lst]
                        d = q - p
                        d -= L * np.round(d / L)
                        if np.any(np.einsum("ij,ij->i", d, d) < d_min * d_min):
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[placed] = p
                cells.setdefault(c, []).append(placed)
                placed += 1
                fails = 0
                if placed == n:
                    break
            else:
                fails += 1
                if fails >= max_tries:
                    raise RuntimeError("rsa_liquid: insertion failed %d times in a row" % fails)
    return pos, box


def maxwell(masses: np.ndarray, T: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (Angstrom/fs) at exactly temperature T.

    v ~ N(0, kB T kappa / m) per component; the centre-of-mass momentum is
    removed and the result rescaled so that sum(m v^2)/(kappa (3N-3) kB) = T.
    """
    n = masses.shape[0]
    z = normal(seed, STREAM_VELOCITY, 3 * n).reshape(n, 3)
    v = z * np.sqrt(KB_EV * T * KAPPA / masses)[:, None]
    p = (masses[:, None] * v).sum(0)
    v -= p / masses.sum()
    ke2 = (masses[:, None] * v * v).sum() / KAPPA       # = 2 KE in eV
    t_now = ke2 / ((3 * n - 3) * KB_EV)
    return v * math.sqrt(T / t_now)


# ----------------------------------------------------------------------------
# Workloads (sizes, densities and seeds of the five benchmark configurations)
# ----------------------------------------------------------------------------

@dataclass
class System:
    pos: np.ndarray          # [N,3] float64, Angstrom
    box: np.ndarray          # [3] float64
    species: np.ndarray      # [N] int32
    masses: np.ndarray       # [N] float64, amu
    name: str = ""
    extra: dict = field(default_factory=dict)


def _fcc_system(cells, a, sigma, seed, species_fracs, species_names, name):
    pos, box = fcc(cells, a)
    if sigma > 0:
        pos = displace(pos, sigma, seed)
    n = pos.shape[0]
    if len(species_fracs) == 1:
        sp = np.zeros(n, dtype=np.int32)
    else:
        sp = assign_species(n, species_fracs, seed)
    masses = np.array([MASS[s] for s in species_names])[sp]
    return System(pos, box, sp, masses, name)


def cu_fcc_small(seed=0) -> System:
    """108-atom FCC Cu, 3x3x3 cells, a = 3.615, sigma = 0.05."""
    return _fcc_system((3, 3, 3), 3.615, 0.05, seed, [1.0], ["Cu"], "fcc-cu-108")


def alloy_fcc(cells=(10, 10, 10), a=3.6, sigma=0.08, seed=1) -> System:
    """Random 50/50 Cu-Ni FCC alloy, default 4,000 atoms."""
    n = 4 * cells[0] * cells[1] * cells[2]
    return _fcc_system(cells, a, sigma, seed, [0.5, 0.5], ["Cu", "Ni"],
                       "fcc-alloy-%d" % n)


def liquid3(n=32_000, density=0.08, d_min=1.8, seed=2) -> System:
    """3-species (Cu/Ni/Al 0.5/0.3/0.2) random liquid-like periodic cube."""
    pos, box = rsa_liquid(n, density, d_min, seed)
    sp = assign_species(n, [0.5, 0.3, 0.2], seed)
    masses = np.array([MASS["Cu"], MASS["Ni"], MASS["Al"]])[sp]
    return System(pos, box, sp, masses, "liquid3-%d" % n)


def cu_fcc_large(cells=(64, 64, 64), sigma=0.0, seed=4) -> System:
    """FCC Cu, a = 3.615; default 64^3 cells = 1,048,576 atoms."""
    n = 4 * cells[0] * cells[1] * cells[2]
    return _fcc_system(cells, 3.615, sigma, seed, [1.0], ["Cu"], "fcc-cu-%d" % n)


def supported_particles(cells_xy=(8, 8), slab_cells=3, radius=6.0, grid=(2, 2), a=3.6,
                        gap=2.0, vacuum=10.0, sigma=0.05, seed=5) -> System:
    """Spherical FCC particles on a planar FCC support slab: a heterogeneous
    geometry like the paper's Pt-TiO2 particles on slabs (Supplementary S1).

    The support (species 0, Ni) is slab_cells FCC cells thick, periodic in x
    and y (box cells_xy * a).  One particle (species 1, Cu) of the given
    radius sits above the centre of each of the grid[0] x grid[1] tiles of
    the xy plane: the FCC sites, with a site at the particle centre, within
    the radius.  Its lowest sites lie ``gap`` above the support's top atomic
    plane; ``vacuum`` separates the particle tops from the support's periodic
    image in z.  Coordinates get N(0, sigma^2) displacements.
    """
    nx, ny = cells_xy
    slab, _ = fcc((nx, ny, slab_cells), a)
    Lx, Ly = nx * a, ny * a
    top = (slab_cells - 0.5) * a                 # highest support plane
    zc = top + gap + radius
    m = int(math.ceil(radius / a)) + 1
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    g = np.arange(-m, m + 1, dtype=np.float64)
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    sites = ((np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)[:, None, :]
              + basis[None]) * a).reshape(-1, 3)
    ball = sites[np.sqrt((sites ** 2).sum(axis=1)) <= radius]
    if 2 * radius + 2.0 > min(Lx / grid[0], Ly / grid[1]):
        raise ValueError("particles would touch: enlarge cells_xy or reduce radius")
    parts = []
    for iy in range(grid[1]):
        for ix in range(grid[0]):
            c = np.array([(ix + 0.5) * Lx / grid[0], (iy + 0.5) * Ly / grid[1], zc])
            parts.append(ball + c)
    part_pos = np.concatenate(parts)
    pos = np.concatenate([slab, part_pos])
    box = np.array([Lx, Ly, zc + radius + vacuum], dtype=np.float64)
    if sigma > 0:
        pos = displace(pos, sigma, seed)
    sp = np.concatenate([np.zeros(len(slab), np.int32), np.ones(len(part_pos), np.int32)])
    masses = np.array([MASS["Ni"], MASS["Cu"]])[sp]
    return System(pos, box, sp, masses, "supported-particles-%d" % len(pos),
                  {"n_support": len(slab), "n_particle_atoms": len(part_pos)})


def model_c1() -> ModelDesc:
    """108-atom case: S=1, F=64, lmax=1, 2 layers, r_c = 5."""
    return ModelDesc(n_species=1, F=64, lmax=1, n_layers_full=2, r_cut=5.0,
                     n_avg=n_avg_for(5.0, 4 / 3.615 ** 3))


def model_alloy(n_layers_full=6) -> ModelDesc:
    """Binary FCC alloy model: S=2, F=128, lmax=2, r_c = 6, a = 3.6."""
    return ModelDesc(n_species=2, F=128, lmax=2, n_layers_full=n_layers_full,
                     r_cut=6.0, n_avg=n_avg_for(6.0, 4 / 3.6 ** 3))


def model_liquid(n_layers_full=6) -> ModelDesc:
    """3-species liquid model at number density 0.08: F=128, lmax=2, r_c = 6."""
    return ModelDesc(n_species=3, F=128, lmax=2, n_layers_full=n_layers_full,
                     r_cut=6.0, n_avg=n_avg_for(6.0, 0.08))


def model_cu(n_layers_full=6, rep_eps=0.0) -> ModelDesc:
    """Large FCC Cu model: S=1, F=128, lmax=2, r_c = 6, a = 3.615."""
    return ModelDesc(n_species=1, F=128, lmax=2, n_layers_full=n_layers_full,
                     r_cut=6.0, n_avg=n_avg_for(6.0, 4 / 3.615 ** 3),
                     rep_eps=rep_eps)
