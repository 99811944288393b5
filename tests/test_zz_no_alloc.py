"""mp_energy_sum_noalloc: the energy sum for callers that cannot allocate
device memory mid-run (pool-managed MD engines), checked through the C ABI
against mp_energy_forces' own FP64 energy on two calls in a row.

Collected last on purpose: a failure here leaves every other test run.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

F32_ENERGY = 1e-6     # |E - E_ref| <= 1e-6 N rms_i(E_i), as in the FP32 energy tests


def test_noalloc_energy_sum_matches_energy_forces(mp):
    s = synth.alloy_fcc(cells=(6, 6, 6), seed=3)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    n = len(s.pos)
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    try:
        e_atom = torch.empty(n, dtype=torch.float64, device="cuda")
        E, _, _ = mp.mp_energy_forces(pot.ctx, pos, sp, g, None, 2, mp.MP_FP32, e_atom=e_atom)
        torch.cuda.synchronize()
        E = float(E.item())
        erms = float(torch.sqrt((e_atom ** 2).mean()).item())
        got = []
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            mp.mp_energy_sum_noalloc(e_atom, out)
            torch.cuda.synchronize()
            got.append(float(out.item()))
            assert abs(got[-1] - E) <= F32_ENERGY * n * erms
        assert got[0] == got[1]
        # sizes beyond the fixed scratch are refused by the C entry point before
        # anything runs (called directly: the Python wrapper never passes an n
        # larger than its tensor)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = mp._lib.mp_energy_sum_noalloc(e_atom.data_ptr(), mp.MP_NOALLOC_MAX_ATOMS + 1,
                                           out.data_ptr(), mp._stream())
        assert rc == -10
        torch.cuda.synchronize()
        assert float(out.item()) == 0.0
    finally:
        mp.mp_graph_free(g)
        pot.close()
