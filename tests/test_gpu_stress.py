"""GPU stress (virial from the hand-written adjoint) against the oracle's
strain derivative, and partitioned against unpartitioned."""
import numpy as np
import pytest
import torch

import synth
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu


def _alloy(cells=(6, 6, 6), seed=4, K=2):
    s = synth.alloy_fcc(cells=cells, sigma=0.1, seed=seed)
    d = synth.model_alloy(n_layers_full=max(K, 1))
    d.rep_eps = 0.3
    return s, d, synth.make_weights(d, 1)


def _gpu(mp, s, d, w, K, precision, **kw):
    pot = mp.Potential(d, w)
    E, F, S = pot.energy_forces_stress(torch.tensor(s.pos, device="cuda"),
                                       torch.tensor(s.species, device="cuda"), s.box, K,
                                       precision, **kw)
    torch.cuda.synchronize()
    out = float(E.item()), F.cpu().numpy().astype(np.float64), S.cpu().numpy()
    pot.close()
    return out


def _ref(s, d, w, K):
    return om.energy_forces_stress(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut),
                                   w, d, K)


@pytest.mark.parametrize("K", [0, 1, 2])
def test_stress_fp32_matches_oracle(mp, K):
    s, d, w = _alloy(K=K)
    E, F, S = _gpu(mp, s, d, w, K, mp.MP_FP32)
    Er, _, Fr, Sr = _ref(s, d, w, K)
    assert np.abs(S - Sr).max() <= 1e-5 * np.abs(Sr).max(), (S, Sr)
    if K > 0:   # (K = 0: the pair forces nearly cancel, F_rms is no scale for them)
        assert np.abs(F - Fr).max() <= 1e-5 * np.sqrt((Fr ** 2).mean())


def test_stress_fp32_lmax1_model(mp):
    s = synth.cu_fcc_small()
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    _, _, S = _gpu(mp, s, d, w, 2, mp.MP_FP32)
    _, _, _, Sr = _ref(s, d, w, 2)
    assert np.abs(S - Sr).max() <= 1e-5 * np.abs(Sr).max(), (S, Sr)


def test_stress_bf16_matches_oracle(mp):
    s, d, w = _alloy()
    _, _, S = _gpu(mp, s, d, w, 2, mp.MP_BF16)
    _, _, _, Sr = _ref(s, d, w, 2)
    assert np.abs(S - Sr).max() <= 1e-2 * np.abs(Sr).max(), (S, Sr)


@pytest.mark.parametrize("precision,mode", [(0, 0), (0, 1), (1, 0)])
def test_partitioned_stress_equals_unpartitioned(mp, precision, mode):
    s, d, w = _alloy(cells=(6, 6, 16), seed=9)
    _, _, S0 = _gpu(mp, s, d, w, 2, precision)
    _, _, S1 = _gpu(mp, s, d, w, 2, precision, n_parts=4, halo_mode=mode)
    assert np.abs(S1 - S0).max() <= 1e-6 * np.abs(S0).max(), (S0, S1)


def test_stress_call_leaves_energy_and_forces_unchanged(mp):
    s, d, w = _alloy(cells=(4, 4, 4))
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    for precision in (mp.MP_FP32, mp.MP_BF16):
        E0, F0, _ = pot.energy_forces(pos, sp, s.box, 2, precision)
        E1, F1, _ = pot.energy_forces_stress(pos, sp, s.box, 2, precision)
        assert E0.item() == E1.item()
        assert torch.equal(F0, F1)
    pot.close()
