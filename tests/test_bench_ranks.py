"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.  Each
rank reports its own time; every rank must see the slowest one, and the
whole-job value counts all ranks' atom-steps."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [120.0, 95.5][rank]
        got = bench.max_over_ranks(ms, world, torch.device("cpu"))
        out[rank] = (got, bench.weak_value(world, 1000, 10, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 120.0
    assert out[0][1] == pytest.approx(2 * 1000 * 10 / 0.120)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, 1, torch.device("cpu")) == 42.0
    assert bench.weak_value(1, 100, 5, 500.0) == pytest.approx(1000.0)
