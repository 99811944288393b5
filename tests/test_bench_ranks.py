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


def test_roofline_accounting():
    """The per-edge work the roofline divides by: the tensor part is the
    three BF16 radial layers (value row, plus the r-tangent row in the
    adjoint), the FP32 part the per-channel epilogue; the node kernels'
    bytes are each array read or written once."""
    import bench
    F, H = 128, 64
    assert bench.edge_tensor_flops("fwd", F, 2, False) == 2 * (8 * H + H * H + H * 5 * F)
    assert bench.edge_tensor_flops("bwd", F, 2, True) == 2 * 2 * (8 * H + H * H + H * 3 * F)
    assert bench.edge_fp32_flops("bwd", F, False) == 170 * F
    assert bench.edge_fp32_flops("fwd", F, True) == 20 * F
    # the BF16 layer-0 adjoint by hidden unit: no third radial layer on the
    # tensor cores, 73 FLOP per hidden unit and edge, and per atom with a
    # nonzero adjoint the 9 x 64 x 128 multiply-adds of V per species
    assert bench.edge_tensor_flops("bwd", F, 2, True, True) == 2 * 2 * (8 * H + H * H)
    assert bench.edge_fp32_flops("bwd", F, True, True) == 73 * H
    assert bench.edge_fp32_flops("bwd", F, True) == 95 * F
    assert bench.v_first_flops(10, 2) == 2 * 9 * H * F * 2 * 10
    row, lm = 4 * F, 4 * F * 8
    # forward, layer 0 of two: read A (9 rows) and h0, write S and h' (9 rows)
    assert bench.node_bytes_per_atom("fwd", True, False) == (row + lm) + row + row + (row + lm)
    # adjoint of the last layer: read dE/dh'_0, S and A_lm, write alpha
    assert bench.node_bytes_per_atom("bwd", False, True) == row + row + lm + (row + lm)
    # the adjoint's FP32 work at the FP32 peak outlasts its BF16 work at the
    # tensor peak, so its roofline bound is the FP32 pipe
    t_tensor = bench.edge_tensor_flops("bwd", F, 2, False) / 1708e12
    t_alu = bench.edge_fp32_flops("bwd", F, False) / (152 * 128 * 2 * 2.07e9)
    assert t_alu > 2 * t_tensor
