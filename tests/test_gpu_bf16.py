"""BF16 tensor-core path (tcgen05 radial MLP) against the FP64 oracle.

BF16 gate: RMSE(F - F_ref) <= 1e-2 F_rms and |E - E_ref| <= 5e-3 N rms_i(E_i);
partitioned vs unpartitioned forces within 1e-6 F_rms (the tensor-core
results of an edge do not depend on which partition holds it).
"""
import numpy as np
import pytest
import torch

import gates
import synth
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu

BF16_FORCE_RMSE = 1e-2
BF16_ENERGY = 5e-3


def _run(mp, d, w, s, K, precision, **kw):
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    E, F, Ei = pot.energy_forces(pos, sp, s.box, K, precision, per_atom=True, **kw)
    torch.cuda.synchronize()
    out = float(E.item()), F.cpu().numpy().astype(np.float64), Ei.cpu().numpy()
    pot.close()
    return out


def _oracle(d, w, s, K):
    return om.energy_forces(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut), w, d, K)


def _check_bf16(got, ref, n):
    E, F, _ = got
    Er, Eir, Fr = ref
    frms = np.sqrt((Fr ** 2).mean())
    rmse = np.sqrt(((F - Fr) ** 2).mean())
    assert rmse <= BF16_FORCE_RMSE * frms, rmse / frms
    erms = np.sqrt((Eir ** 2).mean())
    print("BF16 vs oracle: force RMSE %.3g F_rms, max %.3g F_rms, energy %.3g"
          % (rmse / frms, np.abs(F - Fr).max() / frms, abs(E - Er) / (n * erms)))
    assert abs(E - Er) <= BF16_ENERGY * n * erms, abs(E - Er) / (n * erms)
    return rmse / frms


def test_bf16_c2_4000_pruned(mp):
    s = synth.alloy_fcc()
    d = synth.model_alloy(n_layers_full=6)
    w = synth.make_weights(d, 1)
    _check_bf16(_run(mp, d, w, s, 2, mp.MP_BF16), _oracle(d, w, s, 2), len(s.pos))


def test_bf16_liquid_subcell(mp):
    s = synth.liquid3(n=2000, seed=12)
    d = synth.model_liquid(n_layers_full=2)
    w = synth.make_weights(d, 2)
    _check_bf16(_run(mp, d, w, s, 2, mp.MP_BF16), _oracle(d, w, s, 2), len(s.pos))


@pytest.mark.parametrize("K", [1, 3])
def test_bf16_depths_with_pair_term(mp, K):
    s = synth.alloy_fcc(cells=(5, 5, 5), sigma=0.12, seed=5)
    d = synth.model_alloy(n_layers_full=3)
    d.rep_eps = 0.5
    w = synth.make_weights(d, 1)
    _check_bf16(_run(mp, d, w, s, K, mp.MP_BF16), _oracle(d, w, s, K), len(s.pos))


def test_bf16_four_species(mp):
    """Four species: the hidden-unit layer-0 forward handles up to three, so
    this case runs the channel-wise layer-0 forward beside the hidden-unit
    layer-0 adjoint (whose per-atom vectors V are formed for each of the
    four species)."""
    pos, box = synth.fcc((5, 5, 5), 3.6)
    pos = synth.displace(pos, 0.1, 21)
    sp = synth.assign_species(len(pos), (0.4, 0.3, 0.2, 0.1), 21)
    assert set(np.unique(sp)) == {0, 1, 2, 3}
    s = synth.System(pos, box, sp, np.ones(len(pos)), "alloy4")
    d = synth.model_alloy(n_layers_full=2)
    d.n_species = 4
    w = synth.make_weights(d, 5)
    _check_bf16(_run(mp, d, w, s, 2, mp.MP_BF16), _oracle(d, w, s, 2), len(s.pos))


def test_bf16_close_to_fp32(mp):
    s = synth.alloy_fcc(cells=(6, 6, 6), seed=7)
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 3)
    a = _run(mp, d, w, s, 2, mp.MP_BF16)
    b = _run(mp, d, w, s, 2, mp.MP_FP32)
    frms = np.sqrt((b[1] ** 2).mean())
    assert np.sqrt(((a[1] - b[1]) ** 2).mean()) <= BF16_FORCE_RMSE * frms


@pytest.mark.parametrize("P,mode", [(4, 0), (4, 1)])
def test_bf16_partitioned_equals_unpartitioned(mp, P, mode):
    s = synth.alloy_fcc(cells=(6, 6, 16), sigma=0.1, seed=9)
    d = synth.model_alloy(n_layers_full=2)
    d.rep_eps = 0.3
    w = synth.make_weights(d, 1)
    a = _run(mp, d, w, s, 2, mp.MP_BF16)
    b = _run(mp, d, w, s, 2, mp.MP_BF16, n_parts=P, halo_mode=mode)
    ok, gap = gates.output_gap(b[1], a[1])
    assert ok, gap
    assert np.array_equal(a[2], b[2])
    pot = mp.Potential(d, w)
    pos = torch.tensor(s.pos, device="cuda")
    sp = torch.tensor(s.species, device="cuda")
    f64 = [gates.fp64_forces(mp, pot, pos, sp, s.box, 2, mp.MP_BF16, n_parts=q, halo_mode=mode)
           for q in (1, P)]
    pot.close()
    assert gates.fp64_gap(f64[1], f64[0]) <= gates.GATE, gates.fp64_gap(f64[1], f64[0])


def test_bf16_deterministic(mp):
    s = synth.alloy_fcc(cells=(4, 4, 4))
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    a = _run(mp, d, w, s, 2, mp.MP_BF16)
    b = _run(mp, d, w, s, 2, mp.MP_BF16)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_bf16_unsupported_shape_is_an_error(mp):
    s, d = synth.cu_fcc_small(), synth.model_c1()       # F = 64, lmax = 1
    w = synth.make_weights(d, 0)
    with pytest.raises(mp.MPError) as e:
        _run(mp, d, w, s, 2, mp.MP_BF16)
    assert e.value.code == -8
