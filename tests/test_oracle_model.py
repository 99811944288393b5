"""Oracle network pinned by closed forms, library routines, special cases,
symmetries and finite differences."""
import itertools
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import torch

import synth
from oracle import model as om
from oracle import neighbors as nb


# ------------------------------------------------------------------ basis --

def test_bessel_is_spherical_j0_and_orthonormal():
    rc, nbasis = 6.0, 8
    r = np.linspace(0.3, 5.9, 57)
    e = om.bessel(torch.tensor(r), rc, nbasis).numpy()
    for k in range(1, nbasis + 1):
        z = k * math.pi * r / rc
        ref = math.sqrt(2.0 / rc) * (k * math.pi / rc) * scipy.special.spherical_jn(0, z)
        assert np.allclose(e[:, k - 1], ref, rtol=1e-13, atol=1e-14)
    # orthonormal with weight r^2 on [0, r_c]
    for k, l in itertools.product(range(1, 4), repeat=2):
        f = lambda x: (om.bessel(torch.tensor([x], dtype=torch.float64), rc, nbasis)[0, k - 1]
                       * om.bessel(torch.tensor([x], dtype=torch.float64), rc, nbasis)[0, l - 1]).item() * x * x
        val, _ = scipy.integrate.quad(f, 1e-9, rc, limit=200)
        assert abs(val - (1.0 if k == l else 0.0)) < 1e-8


def test_envelope_smoothness():
    x = torch.tensor([0.0, 1.0], dtype=torch.float64, requires_grad=True)
    u = om.envelope(x, 6)
    assert u[0].item() == 1.0 and abs(u[1].item()) < 1e-15
    # derivatives up to second order vanish at x = 1 (evaluate the polynomial
    # branch just inside the cutoff); at x = 0 the first five vanish.
    xs = torch.tensor([1.0 - 1e-7, 1e-3], dtype=torch.float64, requires_grad=True)
    u = om.envelope(xs, 6)
    g1 = torch.autograd.grad(u.sum(), xs, create_graph=True)[0]
    g2 = torch.autograd.grad(g1.sum(), xs)[0]
    assert abs(g1[0].item()) < 1e-10 and abs(g2[0].item()) < 1e-4
    assert abs(1.0 - u[1].item()) < 30 * 1e-3 ** 6
    assert om.envelope(torch.tensor([1.0, 1.5], dtype=torch.float64), 6).abs().max() == 0.0


# -------------------------------------------------------- spherical harm --

def _unit(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_sph_harm_norm_parity_addition():
    a, b = _unit(200, 1), _unit(200, 2)
    Ya = om.sph_harm(torch.tensor(a), 2)
    Yb = om.sph_harm(torch.tensor(b), 2)
    Yn = om.sph_harm(torch.tensor(-a), 2)
    cos = (a * b).sum(1)
    for l in range(3):
        ya, yb = Ya[l].numpy(), Yb[l].numpy()
        assert np.allclose((ya ** 2).sum(1), 2 * l + 1, atol=1e-13)
        assert np.allclose(Yn[l].numpy(), (-1) ** l * ya, atol=1e-14)
        # addition theorem: sum_m Y_lm(a) Y_lm(b) = (2l+1) P_l(a.b)
        assert np.allclose((ya * yb).sum(1), (2 * l + 1) * scipy.special.eval_legendre(l, cos),
                           atol=1e-12)


def test_sph_harm_orthogonal_on_sphere():
    # Lebedev-free check: Gauss-Legendre in cos(theta) x uniform phi grid.
    xg, wg = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * 2 * np.pi / 24
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wt = (wg[:, None] * np.full_like(ph, 2 * np.pi / 24)).ravel()
    Y = np.concatenate([y.numpy() for y in om.sph_harm(torch.tensor(u), 2)], 1)
    G = (Y * wt[:, None]).T @ Y / (4 * np.pi)
    assert np.allclose(G, np.eye(9), atol=1e-12)


# ----------------------------------------------------------------- dimer --

def _silu(x):
    return x / (1.0 + np.exp(-x))


def _dimer_energy_closed_form(r, w, d):
    """Two atoms of species 0 at distance r, one layer, lmax = 1: every
    quantity is a scalar function of r (h1 = 0 before the layer, and
    B1 = 3 (R1a h0 / N_avg)^2 because sum_m Y1m^2 = 3)."""
    x = r / d.r_cut
    p = d.p_env
    u = 1 - (p + 1) * (p + 2) / 2 * x ** p + p * (p + 2) * x ** (p + 1) - p * (p + 1) / 2 * x ** (p + 2)
    k = np.arange(1, d.n_basis + 1)
    eps = np.sqrt(2 / d.r_cut) * np.sin(k * np.pi * x) / r * u
    R = w["W3"][0] @ _silu(w["W2"][0] @ _silu(w["W1"][0] @ eps))
    F = d.F
    h0 = w["emb"][0]
    A0 = R[:F] * h0 / d.n_avg
    B1 = 3.0 * (R[F:2 * F] * h0 / d.n_avg) ** 2
    s = w["W0"][0] @ A0 + w["U1"][0] @ B1 + w["b"][0]
    return 2.0 * float(w["w_out"] @ (h0 + _silu(s)))


@pytest.mark.parametrize("r", [1.7, 2.5, 3.3, 4.9])
def test_dimer_energy_and_force_closed_form(r):
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    box = np.array([30.0, 30.0, 30.0])
    u = _unit(1, 7)[0]
    pos = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
    e = nb.brute_force_edges(pos, box, d.r_cut)
    assert len(e[0]) == 2
    E, Ei, F = om.energy_forces(pos, np.zeros(2, np.int32), box, e, w, d, 1)
    assert abs(E - _dimer_energy_closed_form(r, w, d)) < 1e-12 * max(1, abs(E))
    h = 1e-5
    dEdr = (_dimer_energy_closed_form(r + h, w, d) - _dimer_energy_closed_form(r - h, w, d)) / (2 * h)
    assert np.allclose(F[1], -dEdr * u, atol=1e-8)
    assert np.allclose(F[0], dEdr * u, atol=1e-8)


# ------------------------------------------------ dimer, any depth, l <= 2 --

def _dimer_energy_recursion(r, w, d, n_layers, z=(0, 1)):
    """Heteronuclear dimer at distance r, any number of layers and lmax <= 2,
    written without spherical harmonics.

    Atom 0 sees its partner along u, atom 1 along -u.  By induction every
    l >= 1 feature stays of the form hl_i[c, m] = a_li[c] Y_lm(u_i): it is
    zero at the start, and a layer adds V_l A_l where A_l[c, m] = beta_li[c]
    Y_lm(u_i), because the partner's Y_lm(u_j) = (-1)^l Y_lm(u_i).  With
    sum_m Y_lm^2 = 2l + 1 every quantity is then a channel vector:
        A0_i   = R0 h0_j / N
        beta_li = (Rla h0_j + (-1)^l Rlb a_lj) / N,  B_li = (2l + 1) beta_li^2
        h0_i  += silu(W0 A0_i + sum_l Ul B_li + b),  a_li += Vl beta_li
    and E = sum_i (w_out . h0_i + e0[z_i])."""
    x = r / d.r_cut
    p = d.p_env
    u = 1 - (p + 1) * (p + 2) / 2 * x ** p + p * (p + 2) * x ** (p + 1) - p * (p + 1) / 2 * x ** (p + 2)
    k = np.arange(1, d.n_basis + 1)
    eps = np.sqrt(2 / d.r_cut) * np.sin(k * np.pi * x) / r * u
    F = d.F
    h0 = [w["emb"][z[0]].copy(), w["emb"][z[1]].copy()]
    a = [[np.zeros(F) for _ in range(d.lmax + 1)] for _ in range(2)]
    for t in range(n_layers):
        R = w["W3"][t] @ _silu(w["W2"][t] @ _silu(w["W1"][t] @ eps))
        new_h0, new_a = [], []
        for i in (0, 1):
            j = 1 - i
            s = w["W0"][t] @ (R[:F] * h0[j] / d.n_avg) + w["b"][t]
            ai = [None]
            for l in range(1, d.lmax + 1):
                Rla = R[(2 * l - 1) * F:(2 * l) * F]
                Rlb = R[(2 * l) * F:(2 * l + 1) * F]
                beta = (Rla * h0[j] + (-1) ** l * Rlb * a[j][l]) / d.n_avg
                s = s + w["U%d" % l][t] @ ((2 * l + 1) * beta ** 2)
                ai.append(a[i][l] + w["V%d" % l][t] @ beta)
            new_h0.append(h0[i] + _silu(s))
            new_a.append(ai)
        h0, a = new_h0, new_a
    return float(sum(w["w_out"] @ h0[i] + w["e0"][z[i]] for i in (0, 1)))


def _dimer_setup(r, n_full=3):
    d = synth.model_alloy(n_layers_full=n_full)
    w = synth.make_weights(d, 3, {"e0": 1.0})
    box = np.array([40.0, 40.0, 40.0])
    u = _unit(1, 11)[0]
    pos = np.array([[15.0, 16.0, 17.0], [15.0, 16.0, 17.0] + r * u])
    return d, w, box, u, pos


@pytest.mark.parametrize("r", [1.9, 2.6, 3.7, 5.3])
def test_dimer_two_and_three_layers_lmax2(r):
    """Layers >= 2 of the lmax = 2 network: the l >= 1 features made by layer
    1 (V_l A_l) enter layer 2's messages through R_lb, and B_2 through U_2.
    Energy to 1e-12 relative, force against the curve's central difference."""
    d, w, box, u, pos = _dimer_setup(r)
    z = np.array([0, 1], np.int32)
    e = nb.brute_force_edges(pos, box, d.r_cut)
    assert len(e[0]) == 2
    for K in (2, 3):
        E, Ei, F = om.energy_forces(pos, z, box, e, w, d, K)
        ref = _dimer_energy_recursion(r, w, d, K)
        assert abs(E - ref) < 1e-12 * max(1.0, abs(E)), (K, E, ref)
        h = 1e-5
        dEdr = (_dimer_energy_recursion(r + h, w, d, K) - _dimer_energy_recursion(r - h, w, d, K)) / (2 * h)
        assert np.allclose(F[1], -dEdr * u, atol=1e-8)
        assert np.allclose(F[0], dEdr * u, atol=1e-8)


def _mutated(w, what):
    m = {k: v.copy() for k, v in w.items()}
    F = m["W0"].shape[-1]
    if what == "V_transposed":
        m["V1"] = np.swapaxes(m["V1"], 1, 2).copy()
        m["V2"] = np.swapaxes(m["V2"], 1, 2).copy()
    elif what == "U2_transposed":
        m["U2"] = np.swapaxes(m["U2"], 1, 2).copy()
    elif what == "R1b_R2a_swapped":
        W3 = m["W3"].copy()
        W3[:, 2 * F:3 * F], W3[:, 3 * F:4 * F] = m["W3"][:, 3 * F:4 * F], m["W3"][:, 2 * F:3 * F]
        m["W3"] = W3
    elif what == "R2b_dropped":
        m["W3"][:, 4 * F:5 * F] = 0.0
    return m


@pytest.mark.parametrize("what", ["V_transposed", "U2_transposed", "R1b_R2a_swapped", "R2b_dropped"])
def test_dimer_recursion_detects_planted_mistakes(what):
    """A mistake planted in the oracle's view of the weights (V_l applied as
    its transpose, U_2 transposed, the R_1b / R_2a slices exchanged, the R_2b
    message dropped) moves the two-layer energy far outside the 1e-12 the
    recursion pins; invariances and finite differences would not see any of
    them."""
    d, w, box, u, pos = _dimer_setup(3.1)
    z = np.array([0, 1], np.int32)
    e = nb.brute_force_edges(pos, box, d.r_cut)
    ref = _dimer_energy_recursion(3.1, w, d, 2)
    E_bad = om.energy(pos, z, box, e, _mutated(w, what), d, 2)
    assert abs(E_bad - ref) > 1e-8 * max(1.0, abs(ref)), (what, E_bad, ref)


# ------------------------------------------------------- special cases --

def test_zero_layers_is_embedding_readout():
    s = synth.alloy_fcc(cells=(4, 4, 4))
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1, {"e0": 1.0})
    e = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E, Ei, F = om.energy_forces(s.pos, s.species, s.box, e, w, d, 0)
    ref = w["emb"][s.species] @ w["w_out"] + w["e0"][s.species]
    assert np.allclose(Ei, ref, atol=1e-14)
    assert np.all(F == 0.0)


def test_perfect_fcc_zero_force_equal_energies():
    pos, box = synth.fcc((4, 4, 4), 3.615)
    d = synth.model_cu(n_layers_full=2)
    w = synth.make_weights(d, 4)
    e = nb.brute_force_edges(pos, box, d.r_cut)
    E, Ei, F = om.energy_forces(pos, np.zeros(len(pos), np.int32), box, e, w, d, 2)
    assert np.abs(F).max() < 1e-11
    assert np.ptp(Ei) < 1e-12 * abs(Ei).max()


def test_supercell_energy_per_atom():
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    vals = []
    for n in (3, 4, 5):
        pos, box = synth.fcc((n, n, n), 3.615)
        e = nb.edges(pos, box, d.r_cut)
        vals.append(om.energy(pos, np.zeros(len(pos), np.int32), box, e, w, d, 2) / len(pos))
    assert np.ptp(vals) < 1e-12 * abs(vals[0])


def test_replication_2x2x2():
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    s = synth.cu_fcc_small()
    e = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E1, _, F1 = om.energy_forces(s.pos, s.species, s.box, e, w, d, 2)
    shifts = np.array(list(itertools.product((0, 1), repeat=3)))[:, ::-1] * s.box
    pos8 = np.concatenate([s.pos + sh for sh in shifts])
    box8 = 2 * s.box
    e8 = nb.edges(pos8, box8, d.r_cut)
    E8, _, F8 = om.energy_forces(pos8, np.zeros(len(pos8), np.int32), box8, e8, w, d, 2)
    assert abs(E8 - 8 * E1) < 1e-11 * abs(E8)
    assert np.allclose(F8, np.tile(F1, (8, 1)), atol=1e-12)


# ---------------------------------------------------------- invariances --

def _c1():
    d = synth.model_c1()
    w = synth.make_weights(d, 0)
    s = synth.cu_fcc_small()
    return s, d, w


def test_translation_invariance():
    s, d, w = _c1()
    e0 = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E0, _, F0 = om.energy_forces(s.pos, s.species, s.box, e0, w, d, 2)
    t = np.array([1.234, -7.77, 3.3])
    p = s.pos + t
    E1, _, F1 = om.energy_forces(p, s.species, s.box, nb.brute_force_edges(p, s.box, d.r_cut), w, d, 2)
    assert abs(E1 - E0) < 1e-12 * abs(E0)
    assert np.allclose(F1, F0, atol=1e-12)


def test_permutation_invariance():
    s, d, w = _c1()
    perm = np.random.default_rng(3).permutation(len(s.pos))
    e0 = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E0, Ei0, F0 = om.energy_forces(s.pos, s.species, s.box, e0, w, d, 2)
    p = s.pos[perm]
    E1, Ei1, F1 = om.energy_forces(p, s.species[perm], s.box,
                                   nb.brute_force_edges(p, s.box, d.r_cut), w, d, 2)
    assert abs(E1 - E0) < 1e-12 * abs(E0)
    assert np.allclose(F1, F0[perm], atol=1e-12)
    assert np.allclose(Ei1, Ei0[perm], atol=1e-13)


def test_cubic_group_invariance_periodic():
    # The 48 signed axis permutations map a periodic cube onto itself.
    s, d, w = _c1()
    L = s.box[0]
    e0 = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E0, _, F0 = om.energy_forces(s.pos, s.species, s.box, e0, w, d, 2)
    ops = list(itertools.product(itertools.permutations(range(3)), itertools.product((1, -1), repeat=3)))
    assert len(ops) == 48
    for perm, sign in ops[::5]:
        R = np.zeros((3, 3))
        for a in range(3):
            R[a, perm[a]] = sign[a]
        p = s.pos @ R.T
        p = p - L * np.floor(p / L)
        E1, _, F1 = om.energy_forces(p, s.species, s.box, nb.brute_force_edges(p, s.box, d.r_cut), w, d, 2)
        assert abs(E1 - E0) < 1e-12 * abs(E0)
        assert np.allclose(F1, F0 @ R.T, atol=1e-12)


def test_arbitrary_rotation_cluster():
    # An isolated cluster in a box much wider than cluster + r_c.
    d = synth.model_alloy(n_layers_full=2)
    w = synth.make_weights(d, 1)
    rng = np.random.default_rng(5)
    pts = []
    while len(pts) < 40:
        p = rng.uniform(-5, 5, 3)
        if np.linalg.norm(p) < 5 and all(np.linalg.norm(p - q) > 1.8 for q in pts):
            pts.append(p)
    pts = np.array(pts)
    sp = (np.arange(40) % 2).astype(np.int32)
    box = np.array([60.0, 60.0, 60.0])
    c = np.array([30.0, 30.0, 30.0])
    E0, _, F0 = om.energy_forces(pts + c, sp, box, nb.brute_force_edges(pts + c, box, d.r_cut), w, d, 2)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    p = pts @ q.T + c
    E1, _, F1 = om.energy_forces(p, sp, box, nb.brute_force_edges(p, box, d.r_cut), w, d, 2)
    assert abs(E1 - E0) < 1e-12 * abs(E0)
    assert np.allclose(F1, F0 @ q.T, atol=1e-11)


# ------------------------------------------------------------ forces FD --

def _fd_check(s, d, w, n_layers, atoms, h=1e-4, tol=1e-7):
    e = nb.brute_force_edges(s.pos, s.box, d.r_cut)
    E, _, F = om.energy_forces(s.pos, s.species, s.box, e, w, d, n_layers)
    assert np.abs(F.sum(0)).max() < 1e-11 * len(s.pos)
    frms = np.sqrt((F ** 2).mean())
    for a in atoms:
        for c in range(3):
            vals = []
            for sgn in (1, -1):
                p = s.pos.copy()
                p[a, c] += sgn * h
                vals.append(om.energy(p, s.species, s.box, nb.brute_force_edges(p, s.box, d.r_cut),
                                      w, d, n_layers))
            fd = -(vals[0] - vals[1]) / (2 * h)
            assert abs(fd - F[a, c]) < tol * max(frms, 1e-3) * 100, (a, c, fd, F[a, c])
    return frms


def test_forces_central_fd_c1():
    s, d, w = _c1()
    _fd_check(s, d, w, 2, atoms=[0, 17, 54, 107])


def test_forces_central_fd_alloy_lmax2_full_depth():
    s = synth.alloy_fcc(cells=(4, 4, 4))
    d = synth.model_alloy(n_layers_full=3)
    d.rep_eps = 0.5
    w = synth.make_weights(d, 1)
    frms = _fd_check(s, d, w, 3, atoms=[3, 200])
    assert 0.05 < frms < 5.0
