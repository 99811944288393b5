"""The partition gate shared by the GPU tests: forces of a partitioned
evaluation against the unpartitioned ones within 1e-6 F_rms (the benchmark
statement's tolerance; the paper states the equality without one).

The library sums each atom's force in FP64, over edges and over partitions,
and rounds it once to FP32 on output.  The gate is applied to those FP64
sums (fp64_forces).  The FP32 outputs are held to the same bound plus one
FP32 spacing of the component (output_gap): two FP64 sums within the bound
can round to neighbouring FP32 values, and one spacing of a component
larger than about 8.4 F_rms already exceeds 1e-6 F_rms."""
import numpy as np
import torch

GATE = 1e-6


def output_gap(F1, F0, gate=GATE):
    """(ok, max |F1 - F0| / F_rms) for FP32 outputs given as float64 arrays."""
    frms = np.sqrt((F0 ** 2).mean())
    spacing = np.spacing(np.abs(F0).astype(np.float32)).astype(np.float64)
    d = np.abs(F1 - F0)
    return bool((d <= gate * frms + spacing).all()), float(d.max() / frms)


def fp64_forces(mp, pot, pos, sp, box, n_layers, precision, n_parts=1, halo_mode=0,
                part=None):
    """FP64 force sums of a K-layer evaluation before their FP32 rounding
    (one partition of the whole system = the unpartitioned evaluation)."""
    g = mp.mp_build_neighbors(pot.ctx, pos, box)
    plan = None
    try:
        if part is not None:
            plan, _ = mp.mp_partition_assign(pot.ctx, g, part, n_parts, n_layers)
        else:
            plan, _ = mp.mp_partition(pot.ctx, g, n_parts, n_layers, halo_mode)
        _, f, _ = mp.mp_energy_forces_parts(pot.ctx, pos, sp, g, plan, 0, n_parts, n_layers,
                                            precision)
        torch.cuda.synchronize()
        return f.cpu().numpy()
    finally:
        if plan:
            mp.mp_plan_free(plan)
        mp.mp_graph_free(g)


def fp64_gap(F1, F0):
    """max |F1 - F0| / F_rms of FP64 force sums."""
    return float(np.abs(F1 - F0).max() / np.sqrt((F0 ** 2).mean()))
