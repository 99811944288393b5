"""Multi-GPU partition distribution: one system, its partitions spread over
the ranks of a process group, one GPU per rank.

The paper runs the subgraphs of a partitioned system as independent forward
passes on several GPUs and gathers their outputs (Introduction, Fig. 1c;
Results, Table 2's GPU x2 / x4 columns): partitions do not communicate during
inference, and the totals are E = sum of root energies and F = sum over
partitions of the gradients of their root energies (Methods, "Global Output
Integration").

Division of work and the exchange per MD step:
  - every rank holds all positions and velocities and builds the same
    neighbour list and partition plan (both deterministic);
  - rank r evaluates the contiguous block of partitions part_range(P, r, W)
    and gets FP64 shares of E and F (mp_energy_forces_parts);
  - one all-reduce (sum) of the FP64 forces [N, 3] and the FP64 energy: the
    reduction of the halo forces across ranks and the energy sum;
  - every rank then applies the same velocity-Verlet halves to all atoms
    (mp_verlet_first_half / mp_verlet_second_half), so the positions stay
    identical on every rank and need no exchange of their own.
An all-reduce gives every rank the same sums, so the replicated state does
not drift apart; ``resync_every`` additionally broadcasts positions and
velocities from rank 0 every so many steps.

The force evaluation and the integrator are the library's kernels
(``LibraryOps``); the collectives are torch.distributed (NCCL on GPUs).  The
orchestration itself takes any object with the same three methods, which is
how the multi-rank logic is tested with gloo on CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def part_range(n_parts: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of partitions of one rank: [begin, end), sizes differing
    by at most one, lower ranks taking the larger blocks."""
    if not (n_parts >= 1 and world >= 1 and 0 <= rank < world):
        raise ValueError("need n_parts >= 1, world >= 1 and 0 <= rank < world")
    base, extra = divmod(n_parts, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


class LibraryOps:
    """Partition evaluation and Verlet halves through the C ABI on this rank's
    GPU (the library's kernels; positions, velocities, masses on the device)."""

    def __init__(self, potential, species, box, n_layers: int, precision: int, n_parts: int,
                 k_hops: int | None = None, halo_mode: int | None = None):
        from . import binding as mp
        self.mp = mp
        self.pot = potential
        self.species = species
        self.box = [float(b) for b in box]
        self.n_layers = n_layers
        self.precision = precision
        self.n_parts = n_parts
        self.k_hops = n_layers if k_hops is None else k_hops
        self.halo_mode = mp.MP_HALO_GEOM if halo_mode is None else halo_mode

    def evaluate_parts(self, pos, begin: int, end: int):
        mp = self.mp
        ctx = self.pot.ctx
        mp.mp_set_stream(ctx, mp._stream())
        g = mp.mp_build_neighbors(ctx, pos, self.box)
        plan = None
        try:
            plan, _ = mp.mp_partition(ctx, g, self.n_parts, self.k_hops, self.halo_mode)
            e, f, _ = mp.mp_energy_forces_parts(ctx, pos, self.species, g, plan, begin, end,
                                                self.n_layers, self.precision)
        finally:
            if plan:
                mp.mp_plan_free(plan)
            mp.mp_graph_free(g)
        return e, f

    def first_half(self, pos, vel, f64, mass, dt: float):
        self.mp.mp_verlet_first_half(self.pot.ctx, pos, vel, f64, mass, self.box, dt)

    def second_half(self, vel, f64, mass, dt: float):
        ke = torch.empty(1, dtype=torch.float64, device=vel.device)
        self.mp.mp_verlet_second_half(self.pot.ctx, vel, f64, mass, dt, ke)
        return ke


class ShardedSystem:
    """Energy, forces and velocity-Verlet MD of one partitioned system whose
    partitions are spread over the ranks of ``group`` (the default group when
    torch.distributed is initialised, else a single rank).

    ``ops`` provides evaluate_parts(pos, begin, end) -> (E [1], F [N, 3]) as
    FP64 shares of partitions begin .. end - 1, first_half(pos, vel, F, m, dt)
    and second_half(vel, F, m, dt) -> KE [1]."""

    def __init__(self, ops, n_parts: int, group=None, resync_every: int = 0):
        self.ops = ops
        self.group = group
        if dist.is_available() and dist.is_initialized():
            self.world = dist.get_world_size(group)
            self.rank = dist.get_rank(group)
        else:
            self.world, self.rank = 1, 0
        self.n_parts = n_parts
        self.parts = part_range(n_parts, self.rank, self.world)
        self.resync_every = resync_every

    def _sum(self, t):
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def energy_forces(self, pos):
        """Totals on every rank: E (FP64 [1]) and F (FP64 [N, 3])."""
        e, f = self.ops.evaluate_parts(pos, *self.parts)
        return self._sum(e), self._sum(f)

    def _resync(self, pos, vel):
        if self.world > 1:
            src = dist.get_global_rank(self.group, 0) if self.group is not None else 0
            dist.broadcast(pos, src, group=self.group)
            dist.broadcast(vel, src, group=self.group)

    def md(self, pos, vel, mass, dt: float, n_steps: int, forces=None):
        """n_steps velocity-Verlet steps in place; returns the final forces (FP64)
        and the ledger [(PE, KE, PE + KE)] after each step (host floats)."""
        if forces is None:
            _, forces = self.energy_forces(pos)
        ledger = []
        for s in range(n_steps):
            self.ops.first_half(pos, vel, forces, mass, dt)
            if self.resync_every and (s + 1) % self.resync_every == 0:
                self._resync(pos, vel)
            e, forces = self.energy_forces(pos)
            ke = self.ops.second_half(vel, forces, mass, dt)
            pe, k = float(e.reshape(-1)[0]), float(ke.reshape(-1)[0])
            ledger.append((pe, k, pe + k))
        return forces, ledger
