"""GPU layer diagnostics (MFS, linear CKA) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import diagnostics as od
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 2e-2)])
def test_layer_stats_match_oracle(mp, precision, tol):
    s = synth.alloy_fcc(cells=(6, 6, 6), sigma=0.1, seed=2)
    d = synth.model_alloy(n_layers_full=4)
    w = synth.make_weights(d, 1)
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    g = mp.mp_build_neighbors(pot.ctx, pos, s.box)
    try:
        m, c = mp.mp_layer_stats(pot.ctx, pos, torch.tensor(s.species, device="cuda"), g, 4,
                                 precision)
    finally:
        mp.mp_graph_free(g)
        pot.close()
    mr, cr = od.layer_stats(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w, d, 4)
    assert np.abs(m - mr).max() <= tol * np.abs(mr).max(), (m, mr)
    assert np.abs(c - cr).max() <= tol * np.abs(1 - cr).max() + 1e-9, (c, cr)
