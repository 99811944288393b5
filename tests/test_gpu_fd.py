"""The hand-written adjoint against central finite differences of the GPU's
own energy, on the 4,000-atom Cu/Ni alloy (10^3 FCC cells, a = 3.6 A,
0.08 A displacements; F = 128, lmax = 2, r_c = 6), 20 seeded atoms, all
three components, FP32 kernels.

Only atoms within K r_c of the displaced atom change their energy, so the
numerator is sum_i (E_i(+h) - E_i(-h)) over the per-atom energies (FP64
copies of FP32 results); every other term is bit-identical in both runs and
cancels exactly.  What remains is FP32 rounding: each changed E_i carries an
error of about sigma_i = |E_i - E_i,oracle| (measured once at the
unperturbed positions), and the +h and -h runs round independently, so the
numerator's noise is about sqrt(2 sum_i sigma_i^2) and the difference
quotient's noise that divided by 2h.  The bound is 6 times that plus the
O(h^2) truncation term (h^2 / 6 times a third derivative of at most
50 eV/A^4 for this potential).  At h = 1e-4 A the FP32 noise dominates; at
h = 1e-3 A the same bound is ten times tighter.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import model as om
from oracle import neighbors as onb

pytestmark = pytest.mark.gpu

THIRD_DERIV_BOUND = 50.0     # eV / A^4, for the truncation term h^2 / 6 |E'''|


def _min_image_dist(pos, box, a):
    d = pos - pos[a]
    d -= box * np.round(d / box)
    return np.sqrt((d * d).sum(1))


@pytest.mark.parametrize("K,n_atoms", [(2, 20), (6, 4)])
def test_adjoint_matches_central_differences_alloy4000(mp, K, n_atoms):
    s = synth.alloy_fcc()
    d = synth.model_alloy(n_layers_full=6)
    w = synth.make_weights(d, 1)
    assert len(s.pos) == 4000
    pot = mp.Potential(d, w)
    sp = torch.tensor(s.species, device="cuda")
    try:
        def run(p):
            E, F, Ei = pot.energy_forces(torch.tensor(p, device="cuda"), sp, s.box, K,
                                         mp.MP_FP32, per_atom=True)
            torch.cuda.synchronize()
            return F.cpu().numpy().astype(np.float64), Ei.cpu().numpy()

        F0, Ei0 = run(s.pos)
        _, Eir, Fr = om.energy_forces(s.pos, s.species, s.box, onb.edges(s.pos, s.box, d.r_cut),
                                      w, d, K)
        sigma = np.abs(Ei0 - Eir)          # FP32 error of each per-atom energy
        frms = float(np.sqrt((Fr ** 2).mean()))
        atoms = synth.seeded_permutation(len(s.pos), 21, 0x0FD)[:n_atoms]
        worst = {}
        for h in (1e-4, 1e-3):
            worst[h] = 0.0
            for a in atoms:
                near = _min_image_dist(s.pos, s.box, a) < K * d.r_cut + 0.5
                noise = np.sqrt(2.0 * (sigma[near] ** 2).sum()) / (2 * h)
                tol = 6.0 * noise + h * h / 6.0 * THIRD_DERIV_BOUND
                for c in range(3):
                    vals = []
                    for sgn in (1, -1):
                        p = s.pos.copy()
                        p[a, c] += sgn * h
                        vals.append(run(p)[1])
                    diff = vals[0] - vals[1]
                    assert np.all(diff[~near] == 0.0)      # untouched atoms cancel exactly
                    fd = -diff[near].sum() / (2 * h)
                    err = abs(fd - F0[a, c])
                    worst[h] = max(worst[h], err / frms)
                    assert err <= tol, (h, a, c, fd, F0[a, c], tol)
        print("K=%d: F_rms %.3f eV/A, max |FD - F| / F_rms = %.2e (h = 1e-4), %.2e (h = 1e-3)"
              % (K, frms, worst[1e-4], worst[1e-3]))
    finally:
        pot.close()
