"""Benchmark: velocity-Verlet MD throughput (atom-steps/s) of the depth-pruned
message-passing potential on one GB300 per rank.

Default workload (N=1): 1,048,576-atom FCC Cu (64^3 cubic cells, a = 3.615 A),
Maxwell velocities at 600 K, pruned K = 2 layers of the 6-layer model (F = 128,
lmax = 2, r_c = 6 A), 8 z-slab partitions with a 12 A geometric halo processed
one after another, dt = 1 fs.  A step is one full MD step: neighbour list,
partitions, energy + forces through the hand-written adjoint, Verlet update.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision bf16|fp32] [--layers K] [--parts P] [--cells n]
                  [--partitioner slabs|graph] [--study partition]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a 6x6x6-cell block of the same lattice and model) on the host cores.
Under torchrun every rank simulates its own independent copy of the system
(no data-path collective, weak scaling); value = all ranks' atom-steps / the
slowest rank's time.  With --shard the ranks instead share the partitions of
one system (the paper's multi-GPU mode): one all-reduce of the FP64 forces
and energy per step, strong scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MD atom-steps/s on 1 GB300 at 32k/1M atoms; force error vs FP64 oracle"
UNIT = "atom-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--layers", type=int, default=2)
    ap.add_argument("--parts", type=int, default=8)
    ap.add_argument("--cells", type=int, default=64, help="FCC cells per axis")
    ap.add_argument("--structure", default="fcc", choices=["fcc", "liquid", "alloy"],
                    help="fcc: FCC Cu (cells^3 x 4 atoms); liquid: 3-species random liquid; "
                         "alloy: random Cu/Ni FCC alloy (a = 3.6 A, 0.08 A displacements)")
    ap.add_argument("--atoms", type=int, default=32000, help="atoms of the liquid")
    ap.add_argument("--partitioner", default="slabs", choices=["slabs", "graph"],
                    help="slabs: z bins with a geometric halo (the benchmark's); graph: roots "
                         "from the multilevel graph partitioner, assigned once, BFS halos")
    ap.add_argument("--shard", action="store_true",
                    help="the paper's multi-GPU mode: under torchrun the ranks share the "
                         "partitions of one system (all-reduce of FP64 forces and energy each "
                         "step; strong scaling) instead of each running its own copy")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet skin in A: neighbours and partitions built with r_c + skin and "
                         "reused until an atom has moved more than skin / 2 (0 = rebuilt every "
                         "step, the benchmark's definition)")
    ap.add_argument("--sample-cells", type=int, default=6,
                    help="cells per axis of the oracle's sample block (FCC kinds; the "
                         "liquid sample has 4 x cells^3 atoms)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--study", default=None, choices=["partition"],
                    help="partition: Stage 1 by spatial grid vs the graph partitioner "
                         "(time, halo factor, cut, balance, MD throughput), one JSON line "
                         "per system, instead of the benchmark line")
    return ap.parse_args()


# DRAM read + write bytes per processed edge of the tensor-core edge adjoint
# (its layer-1 launch, its layer-0 launch and the layer-0 per-atom V that
# runs inside the same timed call), from one ncu capture on 131,072 atoms,
# over the edges of the two launches; scaled by the edges of a launch.  The
# figure belongs to the kernel sources whose hash is stored beside it: once
# those sources change, the line reports traffic null until the counters are
# taken again.
TRAFFIC_BYTES_PER_EDGE_BF16 = {"bwd": (393.3, "fedb9e68d704adca")}
TRAFFIC_SOURCES = ("edge_bf16.cu", "edge_math.cuh", "tc.cuh", "kernels.h", "common.cuh")


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 over the edge kernels' sources."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2509_21694_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def max_over_ranks(ms, world, dev):
    """The slowest rank's time: every rank runs its own copy of the workload
    (no data-path collective), the job is done when the last one is."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, n_atoms, steps, ms_max):
    """Whole-job atom-steps/s: all ranks' atom-steps over the slowest time."""
    return world * n_atoms * steps / (ms_max * 1e-3)


def drift_slope(ledger, n_atoms, dt_fs):
    """Least-squares slope of (E_tot(t) - E_tot(0)) / N over the timed steps,
    in meV/atom/ps."""
    import numpy as np
    if ledger.shape[0] < 2:
        return None
    t = np.arange(ledger.shape[0]) * dt_fs * 1e-3
    y = (ledger[:, 2] - ledger[0, 2]) / n_atoms * 1e3
    return float(np.polyfit(t, y, 1)[0])


def system_and_model(args, cells=None, atoms=None):
    """The benchmark structure (or a smaller block of the same kind) and model."""
    import synth
    if args.structure == "liquid":
        # Cu/Ni/Al 0.5/0.3/0.2 at 0.08 A^-3, 1.8 A minimum distance; the pair
        # term keeps the random packing from collapsing during the MD
        s = synth.liquid3(n=atoms or args.atoms, seed=2)
        d = synth.model_liquid(n_layers_full=6)
        d.rep_eps = 0.3
        w = synth.make_weights(d, 1)
    elif args.structure == "alloy":
        # the depth-comparison alloy: 50/50 Cu/Ni on an FCC lattice
        c = cells or args.cells
        s = synth.alloy_fcc(cells=(c,) * 3)
        d = synth.model_alloy(n_layers_full=6)
        w = synth.make_weights(d, 1)
    else:
        # thermal-scale random displacements (0.05 A) so the start is not a
        # perfectly symmetric lattice
        c = cells or args.cells
        s = synth.cu_fcc_large(cells=(c,) * 3, sigma=0.05, seed=4)
        d = synth.model_cu(n_layers_full=6)
        w = synth.make_weights(d, 4)
    return s, d, w


def kernel_ms(timing):
    """CUDA-event milliseconds per kernel class; layer 0 of the edge kernels
    is included in edge_fwd / edge_bwd and also listed on its own."""
    out = {k: round(v["ms"], 3) for k, v in timing.items() if not k.endswith("_l0")}
    for k in ("edge_fwd", "edge_bwd", "node_fwd", "node_bwd"):
        out[k] = round(timing[k]["ms"] + timing[k + "_l0"]["ms"], 3)
        out[k + "_layer0"] = round(timing[k + "_l0"]["ms"], 3)
    return out


def node_bytes_per_atom(kind: str, first: bool, last: bool, F: int = 128, nlm: int = 9) -> int:
    """Algorithmic DRAM bytes per atom of one node-kernel launch (FP32
    features [n][nlm][F]; every array is read or written once).
    forward: read A (nlm F) and h (F at layer 0, whose l >= 1 inputs are zero
    and not stored, else nlm F), write S (F) and h' (F at the last layer, else
    nlm F).  adjoint: read dE/dh'_0 (F), S (F) and A_lm (l >= 1), write
    alpha (nlm F); then, unless last, read dE/dh'_lm and alpha_lm and write
    alpha_lm (l >= 1)."""
    row, lm = 4 * F, 4 * F * (nlm - 1)
    if kind == "fwd":
        h_in = row if (first or last) else row + lm
        h_out = row if last else row + lm
        return (row + lm) + h_in + row + h_out
    b = row + row + lm + (row + lm)
    if not last:
        b += 3 * lm
    return b


def node_hbm(timing, peak_gbs, K):
    """HBM fraction of the node kernels from the library's CUDA-event timers:
    algorithmic bytes (node_bytes_per_atom x atoms of each launch) over the
    summed kernel time, for layer 0 and the later layers."""
    out = {}
    for kind in ("fwd", "bwd"):
        parts = []
        for key, first in (("node_%s_l0" % kind, True), ("node_" + kind, False)):
            t = timing[key]
            if not t["launches"]:
                continue
            # the later layers' timer holds layers 1..K-1; with K = 2 that is the
            # last layer alone, which is the benchmark's case
            last = (K == 1) if first else True
            parts.append((t["atoms"] * node_bytes_per_atom(kind, first, last), t["ms"]))
        if parts:
            byt = sum(p[0] for p in parts)
            ms = sum(p[1] for p in parts)
            gbs = byt / (ms * 1e-3) / 1e9
            out["node_" + kind] = {"gbs": gbs, "frac": gbs / peak_gbs, "bytes": byt, "ms": ms}
    return out


def workload(args):
    import synth
    s, d, w = system_and_model(args)
    v = synth.maxwell(s.masses, 600.0, 4)
    return s, d, w, v


def n_atoms_of(args):
    return args.atoms if args.structure == "liquid" else 4 * args.cells ** 3


def config_dict(args, n_atoms):
    name = {"liquid": "liquid3-%d-md-600K", "alloy": "fcc-cuni-alloy-%d-md-600K"}.get(
        args.structure, "fcc-cu-%d-md-600K") % n_atoms
    return {"workload": name, "atoms": n_atoms,
            "layers_K": args.layers, "layers_full": 6, "F": 128, "lmax": 2, "r_cut_A": 6.0,
            "partitions": args.parts, "halo_A": 6.0 * args.layers,
            "halo_mode": "geometric" if args.partitioner == "slabs" else "bfs",
            "partitioner": "z-slabs" if args.partitioner == "slabs" else "graph (multilevel)",
            "dt_fs": 1.0, "precision": args.precision,
            "skin_A": args.skin,
            "l2": "inputs larger than L2 (per-partition features >> 129 MB)"}


# -------------------------------------------------------------- clocks --

class Clocks:
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, dev_index=0):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(dev_index):
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- roofline --

# Algorithmic FP32 (CUDA-core) FLOPs per directed edge and channel of the
# BF16 edge kernels' epilogues, counted from the formulas as the kernels
# evaluate them (a multiply-add = 2, a multiply or add = 1):
#   adjoint, layer >= 1 (symmetric pair: both directions of the edge):
#     Y-weighted sums of both sides' adjoints (sk_l, sj_l)           32
#     sender gradient dE/dh_k of the reverse edge                     22
#     dE/dR_q of both directions contracted with dR_q/dr              49
#     dE/dY_lm = R_la (ak_lm hj0 -+ aj_lm hk0), with the harmonics'
#       constant factors folded into R_la                             30
#     dY/du contraction (v, 9 multiply-adds) and the pair-gradient
#       share t u + v / r                                             37
#                                                            total   170
#   adjoint, layer 0 (no l >= 1 inputs), channel-wise (FP32 path):
#     P_lm 24, P.Y 16, dE/dY 10, dR contraction 8, dY/du and pair
#     gradient 37                                              total    95
#   forward, layer >= 1: A0 2, l = 1: 13, l = 2: 21            total    36
#   forward, layer 0:                                          total    20
# (all three radial-MLP layers run on the tensor cores; the first, K = 8,
# as one zero-padded K = 16 MMA, counted at its algorithmic K = 8).
# The BF16 layer-0 adjoint runs by hidden unit instead (its sender features
# are species embeddings, so the channel sums factor through W3): per edge
# and hidden unit, D_lm = Vk -+ Vj 9, sum_lm Y_lm D_lm 16, the dE/dr and
# dE/dY shares 11, dY/du contraction 18, v.u and t 7, the pair-gradient
# share 9 and its addition to the row sum 3: 73; plus, per atom with a
# nonzero adjoint and species s, V = (W3 Emb_s)^T alpha: 9 x 64 x 128
# multiply-adds.
FP32_FLOPS_PER_CHANNEL = {("bwd", False): 170, ("bwd", True): 95,
                          ("fwd", False): 36, ("fwd", True): 20}
BWD0_FLOPS_PER_HIDDEN = 73


def edge_fp32_flops(kind: str, F: int, first: bool, hidden_form: bool = False) -> float:
    if hidden_form and kind == "bwd" and first:
        return float(BWD0_FLOPS_PER_HIDDEN * 64)
    return float(FP32_FLOPS_PER_CHANNEL[(kind, first)] * F)


def v_first_flops(alpha_rows: float, n_species: int, F: int = 128, nlm: int = 9,
                  H: int = 64) -> float:
    """FP32 FLOPs of the per-atom vectors V of the hidden-unit layer-0 adjoint."""
    return 2.0 * nlm * H * F * n_species * alpha_rows


def edge_tensor_flops(kind: str, F: int, lmax: int, first: bool,
                      hidden_form: bool = False) -> float:
    """BF16 tensor-core FLOPs per edge: the three radial-MLP layers (NB x H,
    H x H and H x paths F), for the value row and, in the adjoint, its
    r-tangent row; the hidden-unit layer-0 adjoint runs the first two only."""
    H, NB = 64, 8
    n_paths = (1 + lmax) if first else (1 + 2 * lmax)
    rows = 2 if kind == "bwd" else 1
    last = 0 if (hidden_form and kind == "bwd" and first) else H * n_paths * F
    return 2.0 * rows * (NB * H + H * H + last)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------- our arm --

def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2509_21694_gb300 import build
    build.build()
    from paper_2509_21694_gb300 import binding as mp

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, d, w, v0 = workload(args)
    n = len(s.pos)
    prec = mp.MP_BF16 if args.precision == "bf16" else mp.MP_FP32
    stream = torch.cuda.current_stream()
    ctx = mp.mp_create(d, w)
    mp.mp_set_stream(ctx, stream.cuda_stream)
    pos = torch.tensor(s.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    frc = torch.zeros(n, 3, dtype=torch.float32, device=dev)
    mass = torch.tensor(s.masses, device=dev)
    sp = torch.tensor(s.species, device=dev)
    md = dict(n_layers=args.layers, precision=prec, n_parts=args.parts, k_hops=args.layers,
              halo_mode=mp.MP_HALO_GEOM, skin=args.skin)
    if args.partitioner == "graph" and args.parts > 1:
        # roots assigned once by atom id from the initial graph; the BFS halo
        # is rebuilt every step, so every step stays exact
        g0 = mp.mp_build_neighbors(ctx, pos, s.box)
        part, _ = mp.mp_graph_partition(ctx, g0, args.parts, 0.03, seed=1)
        mp.mp_graph_free(g0)
        md.update(halo_mode=mp.MP_HALO_BFS, part=part)

    # warm-up (also computes the initial forces)
    mp.mp_md_step(ctx, pos, vel, frc, mass, sp, s.box, 1.0, args.warmup, **md)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks()
    mp.mp_timing_enable(ctx, True)
    launches0 = mp.mp_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    list_builds = []
    ledger = mp.mp_md_step(ctx, pos, vel, frc, mass, sp, s.box, 1.0, args.steps,
                           forces_valid=True, builds=list_builds, **md)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop(local)
    launches = mp.mp_kernel_launches() - launches0
    timing = mp.mp_timing_read(ctx)
    mp.mp_timing_enable(ctx, False)
    ms_max = max_over_ranks(t0.elapsed_time(t1), world, dev)
    value = weak_value(world, n, args.steps, ms_max)

    # end-to-end through the C ABI from pinned host buffers: every step copies
    # positions and velocities in, runs one MD step and reads back positions,
    # velocities, forces and the energy ledger.
    e2e = None
    if not args.no_e2e:
        h_pos = torch.tensor(pos.cpu().numpy()).pin_memory()
        h_vel = torch.tensor(vel.cpu().numpy()).pin_memory()
        h_frc = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pos.copy_(h_pos, non_blocking=True)
            vel.copy_(h_vel, non_blocking=True)
            mp.mp_md_step(ctx, pos, vel, frc, mass, sp, s.box, 1.0, 1, forces_valid=True, **md)
            h_pos.copy_(pos, non_blocking=True)
            h_vel.copy_(vel, non_blocking=True)
            h_frc.copy_(frc, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = {"value": weak_value(world, n, args.steps, ems), "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * 3 * 8,
               "d2h_bytes_per_step": 2 * n * 3 * 8 + n * 3 * 4 + 3 * 8}

    # roofline of the dominant kernel class (edge kernels: layer 0 and the
    # later layers are timed separately and counted with their own FLOPs)
    peaks, peak_kind = load_peaks()
    merged = {k: {"ms": timing[k]["ms"] + timing.get(k + "_l0", {"ms": 0.0})["ms"]}
              for k in ("edge_fwd", "edge_bwd")}
    dom = max(("edge_fwd", "edge_bwd", "node_fwd", "node_bwd", "neighbors", "partition"),
              key=lambda k: merged[k]["ms"] if k in merged else timing[k]["ms"])
    roof = None
    if dom in ("edge_fwd", "edge_bwd"):
        kind = "fwd" if dom == "edge_fwd" else "bwd"
        t0, t1 = timing[dom + "_l0"], timing[dom]
        launches_all = t0["launches"] + t1["launches"]
        if launches_all:
            dur = (t0["ms"] + t1["ms"]) / launches_all * 1e-3
            edges_per_launch = (t0["edges"] + t1["edges"]) / launches_all
            mhz = clk.get("sm_mhz") or 2070.0
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            alu_peak = sms * 128 * 2 * mhz * 1e6 / 1e12   # FP32 lanes x 2 FLOP x clock
            if args.precision == "fp32":
                # every FLOP of the FP32 path runs on the CUDA cores: the radial
                # MLP (all three layers) and the epilogue
                flops = sum(t["edges"] * (edge_tensor_flops(kind, 128, 2, first) +
                                          edge_fp32_flops(kind, 128, first))
                            for t, first in ((t0, True), (t1, False))) / launches_all
                achieved = flops / dur / 1e12
                roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                        "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": None,
                        "kernel": "k_edge_" + kind,
                        "peak_note": "FP32: %d SMs x 128 lanes x 2 FLOP x median SM "
                                     "clock %.0f MHz" % (sms, mhz),
                        "flops_per_launch": flops}
            else:
                # two resources: the tensor pipe (radial layers 2 and 3) and the
                # FP32 pipe (radial layer 1 and the per-channel epilogue); the
                # bound is the one whose algorithmic work takes longer at peak
                # layer 0 of the adjoint: hidden-unit form, with its per-atom
                # V (launched inside the same timed call; its atoms are the
                # layer-0 node adjoint's rows)
                tfl = (t0["edges"] * edge_tensor_flops(kind, 128, 2, True, True) +
                       t1["edges"] * edge_tensor_flops(kind, 128, 2, False)) / launches_all
                afl = (t0["edges"] * edge_fp32_flops(kind, 128, True, True) +
                       t1["edges"] * edge_fp32_flops(kind, 128, False)) / launches_all
                if kind == "bwd":
                    afl += v_first_flops(timing["node_bwd_l0"]["atoms"], d.n_species) / launches_all
                tpk = peaks.get("bf16_tflops_sustained", 1700.0)
                src_hash = kernel_source_hash()
                per_edge, measured_on = TRAFFIC_BYTES_PER_EDGE_BF16.get(kind, (None, None))
                current = per_edge is not None and measured_on == src_hash
                traffic = per_edge * edges_per_launch if current else None
                views = {
                    "tensor": {"achieved": tfl / dur / 1e12, "peak": tpk,
                               "frac": tfl / dur / 1e12 / tpk, "flops_per_launch": tfl,
                               "ideal_ms": tfl / (tpk * 1e12) * 1e3,
                               "peak_note": "bf16_tflops_sustained of %s peaks" % peak_kind},
                    "alu": {"achieved": afl / dur / 1e12, "peak": alu_peak,
                            "frac": afl / dur / 1e12 / alu_peak, "flops_per_launch": afl,
                            "ideal_ms": afl / (alu_peak * 1e12) * 1e3,
                            "peak_note": "FP32: %d SMs x 128 lanes x 2 FLOP x median SM "
                                         "clock %.0f MHz" % (sms, mhz)}}
                bound = max(views, key=lambda k: views[k]["ideal_ms"])
                v = views[bound]
                roof = {"bound": bound, "achieved": v["achieved"], "peak": v["peak"],
                        "unit": "TFLOP/s", "frac": v["frac"], "traffic": traffic,
                        "kernel": "k_edge_" + kind, "edges_per_launch": edges_per_launch,
                        "launch_ms": dur * 1e3, "views": views,
                        "kernel_source_hash": src_hash,
                        "traffic_note": ("ncu DRAM bytes per processed edge (131,072-atom "
                                         "capture of these kernel sources) x edges per launch"
                                         if current else
                                         "null: the kernel sources changed since the last "
                                         "ncu capture of DRAM bytes")}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16+fp32" if args.precision == "bf16" else "fp32", "data": "synthetic",
           "config": config_dict(args, n), "e2e": e2e, "gpu_launches": launches,
           "roofline": roof, "clocks": clk,
           "kernel_ms": kernel_ms(timing),
           "hbm_kernels": (node_hbm(timing, peaks.get("hbm_gbs", 6800.0), args.layers)
                           if args.layers == 2 else None),
           "energy_drift_meV_per_atom_ps": drift_slope(ledger, n, 1.0),
           "energy_drift_steps": int(ledger.shape[0]),
           "neighbor_list_builds": list_builds[0],
           "peaks": peak_kind}
    mp.mp_destroy(ctx)
    return out


# ------------------------------------------- sharded system (strong) --

def run_shard(args, rank, world):
    """One system, its partitions spread over the ranks (contiguous slab
    blocks); every step all-reduces the FP64 force and energy shares and
    applies the same Verlet halves on every rank.  value = atoms x steps /
    the slowest rank's time (strong scaling: the total work is fixed)."""
    import torch
    from paper_2509_21694_gb300 import build
    build.build()
    from paper_2509_21694_gb300 import binding as mp
    from paper_2509_21694_gb300.sharded import LibraryOps, ShardedSystem

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, d, w, v0 = workload(args)
    n = len(s.pos)
    prec = mp.MP_BF16 if args.precision == "bf16" else mp.MP_FP32
    stream = torch.cuda.current_stream()
    pot = mp.Potential(d, w)
    mp.mp_set_stream(pot.ctx, stream.cuda_stream)
    pos = torch.tensor(s.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    mass = torch.tensor(s.masses, device=dev)
    sp = torch.tensor(s.species, device=dev)
    sysm = ShardedSystem(LibraryOps(pot, sp, s.box, args.layers, prec, args.parts), args.parts)
    forces, _ = sysm.md(pos, vel, mass, 1.0, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = mp.mp_kernel_launches()
    clocks = Clocks()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    forces, ledger = sysm.md(pos, vel, mass, 1.0, args.steps, forces=forces)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop(local)
    ms_max = max_over_ranks(t0.elapsed_time(t1), world, dev)
    import numpy as np
    cfg = config_dict(args, n)
    cfg["parallelism"] = "partitions %d-%d of %d on rank %d of %d" % (
        sysm.parts[0], sysm.parts[1] - 1, args.parts, rank, world)
    out = {"metric": METRIC, "value": n * args.steps / (ms_max * 1e-3), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "strong",
           "vs_baseline": None, "dtype": "bf16+fp32" if args.precision == "bf16" else "fp32",
           "data": "synthetic", "config": cfg, "e2e": None,
           "gpu_launches": mp.mp_kernel_launches() - launches0, "clocks": clk,
           "energy_drift_meV_per_atom_ps": drift_slope(np.array(ledger), n, 1.0),
           "mode": "shard"}
    pot.close()
    return out


# ------------------------------------------- partitioning study (GPU) --

STUDY_SYSTEMS = {
    # bulk FCC Cu (cells per axis) and Ni-supported Cu particles
    # (cells_xy, support cells, particle radius, particle grid)
    "bulk-32k": ("fcc", 20),
    "bulk-131k": ("fcc", 32),
    "bulk-1M": ("fcc", 64),
    "particles-12k": ("particles", ((24, 24), 4, 12.0, (2, 2))),
    "particles-92k": ("particles", ((48, 48), 8, 18.0, (3, 3))),
    "particles-364k": ("particles", ((64, 64), 16, 26.0, (4, 4))),
}


def run_partition_study(args):
    """Stage 1 compared on bulk and heterogeneous systems (Supplementary S1,
    Figs. S1-S2): the z grid (the benchmark's slabs), a grid along x (in the
    support plane) and the multilevel graph partitioner, each with a K-hop
    BFS halo.  Reports wall time of each partitioning call, the halo growth
    factor H, the edge cut, the largest part over the mean, and the BF16 MD
    throughput with z slabs and with the graph parts."""
    import numpy as np
    import torch
    import synth
    from paper_2509_21694_gb300 import build
    build.build()
    from paper_2509_21694_gb300 import binding as mp

    dev = torch.device("cuda", 0)
    P, K = args.parts, args.layers
    lines = []
    for name, (kind, spec) in STUDY_SYSTEMS.items():
        if kind == "fcc":
            s = synth.cu_fcc_large(cells=(spec,) * 3, sigma=0.05, seed=4)
            d = synth.model_cu(n_layers_full=6)
            w = synth.make_weights(d, 4)
        else:
            cxy, sc, rad, grid = spec
            s = synth.supported_particles(cells_xy=cxy, slab_cells=sc, radius=rad, grid=grid,
                                          seed=5)
            d = synth.model_alloy(n_layers_full=6)
            w = synth.make_weights(d, 1)
        n = len(s.pos)
        ctx = mp.mp_create(d, w)
        stream = torch.cuda.current_stream()
        mp.mp_set_stream(ctx, stream.cuda_stream)
        pos = torch.tensor(s.pos, device=dev)
        g = mp.mp_build_neighbors(ctx, pos, s.box)
        recv, send, _ = mp.mp_graph_export(g)
        recv, send = recv.long(), send.long()

        def describe(part, H, ms):
            a = part.long()
            cut = int((a[recv] != a[send]).sum().item()) // 2
            wts = torch.bincount(a, minlength=P).cpu().numpy()
            return {"H": H, "cut": cut, "max_over_mean": float(wts.max() / (n / P)),
                    "ms": ms}

        def timed(fn):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            return r, (time.perf_counter() - t) * 1e3

        # warm the library's buffers once, then time
        plan, _ = mp.mp_partition(ctx, g, P, K, mp.MP_HALO_BFS)
        mp.mp_plan_free(plan)
        (plan, Hz), ms_z = timed(lambda: mp.mp_partition(ctx, g, P, K, mp.MP_HALO_BFS))
        mp.mp_plan_free(plan)
        x = torch.remainder(pos, torch.tensor(s.box, device=dev))
        zb = torch.clamp((x[:, 2] / s.box[2] * P).floor().int(), max=P - 1).contiguous()
        xb = torch.clamp((x[:, 0] / s.box[0] * P).floor().int(), max=P - 1).contiguous()
        plan, Hx = mp.mp_partition_assign(ctx, g, xb, P, K)
        mp.mp_plan_free(plan)
        mp.mp_graph_partition(ctx, g, P, 0.03, seed=1)
        (gres, ms_g) = timed(lambda: mp.mp_graph_partition(ctx, g, P, 0.03, seed=1))
        part, _ = gres
        plan, Hg = mp.mp_partition_assign(ctx, g, part, P, K)
        mp.mp_plan_free(plan)
        row = {"study": "partition", "system": name, "n_atoms": n, "n_edges": int(recv.numel()),
               "n_parts": P, "k_hops": K,
               "grid_z": describe(zb, Hz, ms_z), "grid_x": describe(xb, Hx, None),
               "graph": describe(part, Hg, ms_g)}
        mp.mp_graph_free(g)

        # MD throughput, BF16, K layers, P partitions: z slabs vs graph parts
        v0 = torch.tensor(synth.maxwell(s.masses, 600.0, 4), device=dev)
        mass = torch.tensor(s.masses, device=dev)
        sp = torch.tensor(s.species, device=dev)
        md_rate = {}
        for label, extra in (("grid_z", dict(halo_mode=mp.MP_HALO_BFS)),
                             ("graph", dict(part=part))):
            p_ = pos.clone()
            v_ = v0.clone()
            f_ = torch.zeros(n, 3, dtype=torch.float32, device=dev)
            common = dict(n_layers=K, precision=mp.MP_BF16, n_parts=P, k_hops=K)
            mp.mp_md_step(ctx, p_, v_, f_, mass, sp, s.box, 1.0, 2, **common, **extra)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mp.mp_md_step(ctx, p_, v_, f_, mass, sp, s.box, 1.0, args.steps, forces_valid=True,
                          **common, **extra)
            e1.record(stream)
            torch.cuda.synchronize()
            md_rate[label] = n * args.steps / (e0.elapsed_time(e1) * 1e-3)
        row["md_atom_steps_per_s"] = md_rate
        mp.mp_destroy(ctx)
        print(json.dumps(row), flush=True)
        lines.append(row)
    return lines


# ------------------------------------------------------ oracle (CPU) --

def oracle_sample_step(args, cells=6):
    """One FP64 oracle MD step on a cells^3 block of the same lattice and
    model (FCC), or an independently generated 864-atom cell of the liquid."""
    import synth
    from oracle import md as omd, model as om, neighbors as onb
    s, d, w = system_and_model(args, cells=cells, atoms=4 * cells ** 3)
    v = synth.maxwell(s.masses, 600.0, 4)

    def force(p):
        E, _, F = om.energy_forces(p, s.species, s.box, onb.edges(p, s.box, d.r_cut), w, d,
                                   args.layers)
        return E, F
    state = {"pos": s.pos, "vel": v, "F": force(s.pos)[1]}

    def step():
        p, vv, F, _ = omd.verlet(state["pos"], state["vel"], s.masses, s.box, force, 1.0, 1,
                                 forces=state["F"])
        state.update(pos=p, vel=vv, F=F)
    return len(s.pos), step


def cpu_baseline(args, cells=6, steps=3, warmup=1):
    """The oracle's MD throughput on a bounded sample, timed in a fresh
    process (started with spawn, so it inherits nothing of this process's GPU
    state or thread settings), all host cores after a warm-up step, then one
    step on a single thread."""
    import multiprocessing as mpr
    with mpr.get_context("spawn").Pool(1) as pool:
        return pool.apply(_cpu_baseline_child, (vars(args), cells, steps, warmup))


def _cpu_baseline_child(argd, cells, steps, warmup):
    args = argparse.Namespace(**argd)
    import torch
    threads = os.cpu_count() or 1
    torch.set_num_threads(threads)
    n, step = oracle_sample_step(args, cells)
    for _ in range(warmup):
        step()
    t = time.perf_counter()
    for _ in range(steps):
        step()
    dt = time.perf_counter() - t
    torch.set_num_threads(1)
    t = time.perf_counter()
    step()
    dt1 = time.perf_counter() - t
    torch.set_num_threads(threads)
    return {"value": n * steps / dt, "unit": UNIT, "cores": threads,
            "kind": "oracle", "value_1_thread": n / dt1,
            "sample": "%d-atom %s of the same kind and model (the per-atom rate of a "
                      "linear-scaling method, measured at %d atoms), K=%d, %d warm-up + %d "
                      "timed MD step(s) on %d threads, then 1 step on 1 thread, FP64 torch CPU"
                      % (n, sample_kind(args, cells), n, args.layers, warmup, steps, threads)}


def sample_kind(args, cells):
    if args.structure == "liquid":
        return "liquid cell"
    return ("FCC Cu/Ni alloy block (%d^3 cells)" if args.structure == "alloy"
            else "FCC Cu block (%d^3 cells)") % cells


def run_reference(args):
    import torch
    torch.set_num_threads(os.cpu_count() or 1)
    n, step = oracle_sample_step(args, cells=args.sample_cells)
    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    value = n * args.steps / dt
    # the line carries this arm's config (the benchmark workload); each timed
    # step is a bounded sample of it, which the sample string states
    cb = {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
          "sample_atoms": n,
          "sample": "each step: one FP64 oracle MD step of a %d-atom %s of the same kind and "
                    "model (the per-atom rate, measured at %d atoms, stands for the %d-atom "
                    "workload), K=%d, torch CPU" % (n, sample_kind(args, args.sample_cells), n,
                                                    n_atoms_of(args), args.layers)}
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, n_atoms_of(args)),
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.study == "partition":
        run_partition_study(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if args.shard:
        out = run_shard(args, rank, world)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, cells=6)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
