"""Parity at the benchmark's full size, in the launch configuration bench.py
times (1,048,576 FCC Cu atoms, K = 2, 8 z-slabs with 12 A geometric halos),
on sampled atoms the oracle computes exactly from local clusters; and the
partitioned-vs-unpartitioned check on the 262,144-atom cell."""
import numpy as np
import pytest
import torch

import gates
import synth
from oracle import partition as op

pytestmark = pytest.mark.gpu

SAMPLES = [12345, 700001]


@pytest.fixture(scope="module")
def big():
    s = synth.cu_fcc_large(cells=(64, 64, 64), sigma=0.05, seed=4)
    d = synth.model_cu(n_layers_full=6)
    w = synth.make_weights(d, 4)
    return s, d, w


def _gpu(mp, s, d, w, precision, parts):
    pot = mp.Potential(d, w)
    E, F, Ei = pot.energy_forces(torch.tensor(s.pos, device="cuda"),
                                 torch.tensor(s.species, device="cuda"), s.box, 2, precision,
                                 n_parts=parts, per_atom=True)
    torch.cuda.synchronize()
    out = F.cpu().numpy().astype(np.float64), Ei.cpu().numpy()
    pot.close()
    return out


def test_fullsize_sampled_atoms_fp32_and_bf16(mp, big):
    s, d, w = big
    F32, E32 = _gpu(mp, s, d, w, mp.MP_FP32, 8)
    F16, E16 = _gpu(mp, s, d, w, mp.MP_BF16, 8)
    frms = np.sqrt((F32 ** 2).mean())
    erms = np.sqrt((E32 ** 2).mean())
    for k in SAMPLES:
        Ek, Fk = op.local_energy_force(s.pos, s.species, s.box, w, d, 2, k)
        # FP32 gate per component; BF16: 5x the RMSE gate for a single atom
        assert np.abs(F32[k] - Fk).max() <= 1e-5 * frms, (k, F32[k], Fk)
        assert abs(E32[k] - Ek) <= 1e-6 * erms
        assert np.abs(F16[k] - Fk).max() <= 5e-2 * frms, (k, F16[k], Fk)
        assert abs(E16[k] - Ek) <= 5e-3 * erms
    # whole-system invariants at full size
    assert np.abs(F32.sum(0)).max() <= 1e-6 * frms * len(F32)
    assert np.sqrt(((F16 - F32) ** 2).mean()) <= 1e-2 * frms


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_262k_partitioned_equals_unpartitioned(mp, precision):
    s = synth.cu_fcc_large(cells=(32, 32, 64), sigma=0.05, seed=5)
    d = synth.model_cu(n_layers_full=6)
    w = synth.make_weights(d, 4)
    p = mp.MP_FP32 if precision == "fp32" else mp.MP_BF16
    F1, E1 = _gpu(mp, s, d, w, p, 1)
    F8, E8 = _gpu(mp, s, d, w, p, 8)
    ok, gap = gates.output_gap(F8, F1)
    assert ok, gap
    assert np.array_equal(E1, E8)
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    f64 = [gates.fp64_forces(mp, pot, pos, sp, s.box, 2, p, n_parts=q) for q in (1, 8)]
    pot.close()
    assert gates.fp64_gap(f64[1], f64[0]) <= gates.GATE, gates.fp64_gap(f64[1], f64[0])
