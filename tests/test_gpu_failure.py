"""Failure detection without a GPU fault: a bounded wait that runs out is
reported as MP_ERR_TIMEOUT through the context's error word, and the context
keeps working afterwards."""
import numpy as np
import pytest
import torch

import synth
from oracle import model as om, neighbors as onb

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(mp):
    s = synth.cu_fcc_small()
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    pot = mp.Potential(d, w)
    try:
        # an mbarrier nothing arrives at: the wait gives up after ~1e5 cycles
        assert mp.mp_wait_selftest(pot.ctx, 100_000, arrive=False) == mp.MP_ERR_TIMEOUT
        # the same wait with one arrival succeeds
        assert mp.mp_wait_selftest(pot.ctx, 100_000, arrive=True) == mp.MP_OK
        assert mp.mp_wait_selftest(pot.ctx, 100_000, arrive=False) == mp.MP_ERR_TIMEOUT
        with pytest.raises(mp.MPError) as e:
            mp.mp_wait_selftest(pot.ctx, 0, arrive=False)
        assert e.value.code == mp.MP_ERR_ARG
        # the context (stream, error word, tensor memory) is still usable: a
        # normal evaluation runs and matches the oracle
        E, F, _ = pot.energy_forces(torch.tensor(s.pos, device="cuda"),
                                    torch.tensor(s.species, device="cuda"), s.box, n_layers=2)
        torch.cuda.synchronize()
        Er, _, Fr = om.energy_forces(s.pos, s.species, s.box,
                                     onb.brute_force_edges(s.pos, s.box, d.r_cut), w, d, 2)
        frms = float(np.sqrt((Fr ** 2).mean()))
        assert np.abs(F.cpu().numpy() - Fr).max() <= 1e-5 * frms
        assert abs(float(E.item()) - Er) <= 1e-6 * abs(Er)
    finally:
        pot.close()
