"""The message-passing potential in float64 torch, forces by autograd (oracle;
test infrastructure only).

The paper treats the backbone as a black box of M message-passing layers
whose per-atom energies sum to E (Methods, "Message Passing Depth Pruning"
and "Global Output Integration": E = sum_i E_i, F = -grad E).  The concrete
network below is the reading this project fixes for that black box; every
formula is written out once here, in the order it is applied:

radial basis, x = r / r_c
  e_k(r)   = sqrt(2 / r_c) sin(k pi x) / r,          k = 1..n_basis
  u(x)     = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2),  x < 1
  eps_k    = e_k(r) u(x)
radial MLP of layer t (bias free, sigma = SiLU)
  R        = W3 sigma(W2 sigma(W1 eps)),  R = [R0 | R1a | R1b | R2a | R2b]
real spherical harmonics of u = d / r, component normalisation
  Y0 = 1;  Y1 = sqrt3 (x, y, z)
  Y2 = (sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2 - 1), sqrt15 xz, sqrt15/2 (x^2 - y^2))
messages summed by receiver i over edges e = (i <- j)
  A0_i[c]     = 1/N_avg sum_e R0[c] h0_j[c]
  Al_i[c, m]  = 1/N_avg sum_e (Rla[c] h0_j[c] Y_lm + Rlb[c] hl_j[c, m])
  Bl_i[c]     = sum_m Al_i[c, m]^2
node update
  h0_i <- h0_i + sigma(W0 A0_i + sum_l Ul Bl_i + b)
  hl_i <- hl_i + Vl Al_i       (Vl acts on channels, shared over m)
initial state and readout
  h0 = Emb[z_i], hl = 0;  E_i = w_out . h0_i^(K) + e0[z_i] + E_rep,i
  E_rep,i = 1/2 sum_e eps_rep (sigma_rep / r)^12 u(x)   (optional pair term)
pruning: a K-layer evaluation uses layers 1..K of the L_full weight set and
the same readout.

stress (energy_forces_stress)
  sigma = (1/V) dE/d(eps) for the homogeneous strain d_e -> (I + eps) d_e

Parity pins (tests/test_oracle_*.py): Bessel and envelope closed forms and
envelope derivatives at x = 1, spherical-harmonic norms, parity and addition
theorem, the analytic dimer energy curve, a heteronuclear dimer through two
and three lmax = 2 layers written as a channel-vector recursion (pins
R_lb h^l_j, V_l, U_2 and the R slice order), pairs beyond r_c adding
nothing (the Verlet-skin reading), K = 0 special case, translation /
rotation / permutation invariance, perfect-FCC zero forces, supercell
replication, sum F = 0 and central finite differences of the energy; for the
stress: central differences over real rescalings of the cell, the closed-form
pair-potential virial, symmetry, and the partition sum.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .neighbors import wrap, decode_shift

_T = torch.float64


def silu(x):
    return x * torch.sigmoid(x)


def bessel(r, r_cut: float, n_basis: int):
    k = torch.arange(1, n_basis + 1, dtype=_T)
    return math.sqrt(2.0 / r_cut) * torch.sin(k * math.pi * r[:, None] / r_cut) / r[:, None]


def envelope(x, p: int = 6):
    u = (1.0 - (p + 1) * (p + 2) / 2.0 * x ** p + p * (p + 2) * x ** (p + 1)
         - p * (p + 1) / 2.0 * x ** (p + 2))
    return torch.where(x < 1.0, u, torch.zeros_like(u))


def sph_harm(u, lmax: int):
    """List [Y0 [E,1], Y1 [E,3], Y2 [E,5]] up to lmax, component normalisation."""
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    out = [torch.ones_like(x)[:, None]]
    if lmax >= 1:
        out.append(math.sqrt(3.0) * u)
    if lmax >= 2:
        s15 = math.sqrt(15.0)
        out.append(torch.stack([s15 * x * y, s15 * y * z,
                                math.sqrt(5.0) / 2.0 * (3.0 * z * z - 1.0),
                                s15 * x * z, s15 / 2.0 * (x * x - y * y)], dim=1))
    return out


def _t(a):
    if isinstance(a, torch.Tensor):
        return a
    return torch.as_tensor(np.asarray(a), dtype=_T)


def atom_energies(pos_t, species, box, recv, send, code, w, desc, n_layers,
                  use_head=False, collect=None, strain=None, layer_masks=None):
    """Per-atom energies E_i (torch float64 [N]) as a differentiable function
    of pos_t; recv/send/code is the edge list of these positions.  With
    ``strain`` (a 3 x 3 tensor eps) every edge vector is deformed as
    d -> (I + eps) d, which is what a homogeneous strain of positions and box
    does to it (the edge set itself does not change under an infinitesimal
    strain).  With ``layer_masks`` (one boolean array over the edges per
    layer) layer t sums messages over the edges of mask t only."""
    F, lmax = desc.F, desc.lmax
    N = pos_t.shape[0]
    recv_t = torch.as_tensor(recv, dtype=torch.long)
    send_t = torch.as_tensor(send, dtype=torch.long)
    shift = _t(decode_shift(code)) * _t(box)
    species_t = torch.as_tensor(species, dtype=torch.long)

    d = pos_t[send_t] - pos_t[recv_t] + shift
    if strain is not None:
        d = d @ (torch.eye(3, dtype=_T) + strain).T
    r = torch.sqrt((d * d).sum(1))
    x = r / desc.r_cut
    env = envelope(x, desc.p_env)
    eps = bessel(r, desc.r_cut, desc.n_basis) * env[:, None]
    Y = sph_harm(d / r[:, None], lmax)

    h0 = _t(w["emb"])[species_t]
    hl = [None] + [torch.zeros(N, F, 2 * l + 1, dtype=_T) for l in range(1, lmax + 1)]
    if collect is not None:
        collect.append(h0)
    for t in range(n_layers):
        W1, W2, W3 = _t(w["W1"][t]), _t(w["W2"][t]), _t(w["W3"][t])
        R = silu(silu(eps @ W1.T) @ W2.T) @ W3.T
        if layer_masks is not None:
            R = R * _t(np.asarray(layer_masks[t], dtype=np.float64))[:, None]
        h0j = h0[send_t]
        A0 = torch.zeros(N, F, dtype=_T).index_add(0, recv_t, R[:, :F] * h0j) / desc.n_avg
        s = A0 @ _t(w["W0"][t]).T + _t(w["b"][t])
        newl = [None]
        for l in range(1, lmax + 1):
            Rla = R[:, (2 * l - 1) * F:(2 * l) * F]
            Rlb = R[:, (2 * l) * F:(2 * l + 1) * F]
            msg = (Rla * h0j)[:, :, None] * Y[l][:, None, :] + Rlb[:, :, None] * hl[l][send_t]
            Al = torch.zeros(N, F, 2 * l + 1, dtype=_T).index_add(0, recv_t, msg) / desc.n_avg
            Bl = (Al * Al).sum(-1)
            s = s + Bl @ _t(w["U%d" % l][t]).T
            newl.append(hl[l] + torch.einsum("dc,ncm->ndm", _t(w["V%d" % l][t]), Al))
        h0 = h0 + silu(s)
        hl = newl
        if collect is not None:
            collect.append(h0)
    E = h0 @ _t(w["w_out"]) + _t(w["e0"])[species_t]
    if desc.rep_eps != 0.0:
        pair = desc.rep_eps * (desc.rep_sigma / r) ** 12 * env
        E = E + 0.5 * torch.zeros(N, dtype=_T).index_add(0, recv_t, pair)
    if use_head:
        E = E + head_energy(h0, w)
    return E


def head_energy(h0, w):
    """Correction head E_i^head = W2 . sigma(W1 h0_i + b1) + b2."""
    a = silu(h0 @ _t(w["head_W1"]).T + _t(w["head_b1"]))
    return a @ _t(w["head_W2"]) + _t(w["head_b2"])[0]


def energy_forces(pos, species, box, edges, w, desc, n_layers, seed_mask=None,
                  use_head=False, layer_masks=None):
    """(E, E_i, F) in float64 numpy.

    E = sum_i s_i E_i with s_i = seed_mask (1 for all atoms by default);
    F = -dE/dpos by reverse-mode autograd.  ``edges`` = (recv, send, code)
    computed from the same positions.
    """
    box = np.asarray(box, dtype=np.float64)
    pos_w = wrap(np.asarray(pos, dtype=np.float64), box)
    pos_t = torch.tensor(pos_w, dtype=_T, requires_grad=True)
    recv, send, code = edges
    Ei = atom_energies(pos_t, species, box, recv, send, code, w, desc, n_layers,
                       use_head=use_head, layer_masks=layer_masks)
    if seed_mask is None:
        E = Ei.sum()
    else:
        E = (Ei * _t(seed_mask)).sum()
    if not E.requires_grad:                 # zero layers: E is position independent
        return float(E), Ei.detach().numpy(), np.zeros_like(pos_w)
    (g,) = torch.autograd.grad(E, pos_t)
    return float(E.detach()), Ei.detach().numpy(), -g.numpy()


def energy_forces_stress(pos, species, box, edges, w, desc, n_layers, seed_mask=None,
                         use_head=False):
    """(E, E_i, F, sigma) in float64 numpy.

    sigma = (1 / V) dE/d(eps) at eps = 0 (3 x 3, eV / A^3): the derivative of
    the energy with respect to a homogeneous strain of positions and box,
    taken by reverse-mode autograd through the deformed edge vectors
    (Methods, "Global Output Integration": stress decomposes over the
    per-atom energies like the forces).  E, E_i, F as in energy_forces.
    """
    box = np.asarray(box, dtype=np.float64)
    pos_w = wrap(np.asarray(pos, dtype=np.float64), box)
    pos_t = torch.tensor(pos_w, dtype=_T, requires_grad=True)
    eps = torch.zeros(3, 3, dtype=_T, requires_grad=True)
    recv, send, code = edges
    Ei = atom_energies(pos_t, species, box, recv, send, code, w, desc, n_layers,
                       use_head=use_head, strain=eps)
    E = Ei.sum() if seed_mask is None else (Ei * _t(seed_mask)).sum()
    vol = float(np.prod(box))
    if not E.requires_grad:
        return float(E), Ei.detach().numpy(), np.zeros_like(pos_w), np.zeros((3, 3))
    gp, ge = torch.autograd.grad(E, [pos_t, eps], allow_unused=True)
    F = np.zeros_like(pos_w) if gp is None else -gp.numpy()
    sig = np.zeros((3, 3)) if ge is None else ge.numpy() / vol
    return float(E.detach()), Ei.detach().numpy(), F, sig


def energy(pos, species, box, edges, w, desc, n_layers, use_head=False):
    """Total energy only (no autograd graph)."""
    box = np.asarray(box, dtype=np.float64)
    with torch.no_grad():
        pos_t = torch.tensor(wrap(np.asarray(pos, dtype=np.float64), box), dtype=_T)
        recv, send, code = edges
        return float(atom_energies(pos_t, species, box, recv, send, code, w, desc,
                                   n_layers, use_head=use_head).sum())


def layer_features(pos, species, box, edges, w, desc, n_layers):
    """Scalar node features h0 after every layer, [n_layers + 1] x [N, F]."""
    box = np.asarray(box, dtype=np.float64)
    feats = []
    with torch.no_grad():
        pos_t = torch.tensor(wrap(np.asarray(pos, dtype=np.float64), box), dtype=_T)
        recv, send, code = edges
        atom_energies(pos_t, species, box, recv, send, code, w, desc, n_layers,
                      collect=feats)
    return [f.numpy() for f in feats]
