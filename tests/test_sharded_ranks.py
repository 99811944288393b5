"""The multi-GPU partition distribution's host logic on CPU: two gloo ranks
share the partitions of one system, all-reduce their FP64 shares of E and F,
and integrate the same velocity-Verlet steps.  The per-partition shares come
from the oracle here (each rank's partitions evaluated with root-only
seeding), so the test checks the division of work and the exchange: the
assembled E and F equal the oracle's unpartitioned result, both ranks hold
bit-identical totals and trajectories, and the trajectory equals the
single-process Verlet run."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import synth
from oracle import md as omd
from oracle import model as om
from oracle import neighbors as onb
from oracle import partition as op
from paper_2509_21694_gb300.sharded import ShardedSystem, part_range

K = 2
N_PARTS = 4


def _system():
    s = synth.cu_fcc_small(seed=3)
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    v = synth.maxwell(s.masses, 600.0, 5)
    return s, d, w, v


class OracleOps:
    """CPU stand-in for the library's kernels: FP64 shares of a range of
    partitions (BFS halos of K hops) and the two Verlet halves."""

    def __init__(self, s, d, w):
        self.s, self.d, self.w = s, d, w

    def evaluate_parts(self, pos, begin, end):
        s, d = self.s, self.d
        p = pos.numpy()
        e = onb.edges(p, s.box, d.r_cut)
        parts, _ = op.plan(p, s.box, e, N_PARTS, K, d.r_cut, mode="bfs")
        E, _, F = op.partitioned_energy_forces(p, s.species, s.box, e, self.w, d, K,
                                               parts[begin:end])
        return torch.tensor([E], dtype=torch.float64), torch.tensor(F)

    def first_half(self, pos, vel, f, m, dt):
        vel += 0.5 * dt * synth.KAPPA * f / m[:, None]
        pos += dt * vel
        box = torch.tensor(self.s.box)
        pos -= box * torch.floor(pos / box)

    def second_half(self, vel, f, m, dt):
        vel += 0.5 * dt * synth.KAPPA * f / m[:, None]
        return torch.tensor([0.5 * float((m[:, None] * vel * vel).sum()) / synth.KAPPA],
                            dtype=torch.float64)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, d, w, v = _system()
        sysm = ShardedSystem(OracleOps(s, d, w), N_PARTS)
        pos = torch.tensor(s.pos)
        E, F = sysm.energy_forces(pos)
        vel = torch.tensor(v)
        m = torch.tensor(s.masses)
        F2, ledger = sysm.md(pos, vel, m, 1.0, 3, forces=F.clone())
        out[rank] = dict(parts=sysm.parts, E=float(E[0]), F=F.numpy(), pos=pos.numpy(),
                         vel=vel.numpy(), ledger=np.array(ledger))
    finally:
        dist.destroy_process_group()


def test_part_range_covers_partitions_contiguously():
    for n_parts in (1, 4, 7, 8, 13):
        for world in (1, 2, 3, 4, 8):
            if world > n_parts:
                continue
            ranges = [part_range(n_parts, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n_parts
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        part_range(4, 2, 2)


def test_two_gloo_ranks_assemble_the_unpartitioned_result():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0["parts"] == (0, 2) and r1["parts"] == (2, 4)
    # every rank holds the same totals and the same trajectory, bit for bit
    for key in ("F", "pos", "vel", "ledger"):
        assert np.array_equal(r0[key], r1[key]), key
    assert r0["E"] == r1["E"]
    # the totals are the unpartitioned oracle result
    s, d, w, v = _system()
    e = onb.edges(s.pos, s.box, d.r_cut)
    E_ref, _, F_ref = om.energy_forces(s.pos, s.species, s.box, e, w, d, K)
    frms = np.sqrt((F_ref ** 2).mean())
    assert abs(r0["E"] - E_ref) <= 1e-11 * abs(E_ref)
    assert np.abs(r0["F"] - F_ref).max() <= 1e-11 * frms

    # and the trajectory is the single-process Verlet run
    def force(p):
        E, _, F = om.energy_forces(p, s.species, s.box, onb.edges(p, s.box, d.r_cut), w, d, K)
        return E, F
    pos, vel, _, ledger = omd.verlet(s.pos, v, s.masses, s.box, force, 1.0, 3, forces=F_ref)
    assert np.abs(r0["pos"] - pos).max() <= 1e-10
    assert np.abs(r0["vel"] - vel).max() <= 1e-10
    assert np.allclose(r0["ledger"], ledger, rtol=1e-11, atol=1e-11)


def test_single_rank_without_process_group():
    s, d, w, v = _system()
    sysm = ShardedSystem(OracleOps(s, d, w), N_PARTS)
    assert sysm.world == 1 and sysm.parts == (0, N_PARTS)
    E, F = sysm.energy_forces(torch.tensor(s.pos))
    e = onb.edges(s.pos, s.box, d.r_cut)
    E_ref, _, F_ref = om.energy_forces(s.pos, s.species, s.box, e, w, d, K)
    assert abs(float(E[0]) - E_ref) <= 1e-11 * abs(E_ref)
    assert np.abs(F.numpy() - F_ref).max() <= 1e-11 * np.sqrt((F_ref ** 2).mean())
