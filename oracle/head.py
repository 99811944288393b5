"""Correction-head loss and its gradient in FP64 (oracle; test
infrastructure only).

The learned part of the method as read here: a per-atom head
E_i^head = w2 . silu(W1 h0_i^(K) + b1) + b2 on the pruned model's final scalar
features, trained with the backbone frozen on energies and forces of a
reference model.  Loss of one snapshot of N atoms:

    L = ((E - E_ref) / N)^2 + lambda / (3N) sum_k |F_k - F_ref,k|^2

with E, F the student's energy and forces (F = -dE/dr).  The gradient with
respect to the head parameters is taken by reverse mode twice (through the
force), so it shares nothing with the GPU's forward-mode construction.

Parity pins (tests/test_oracle_head.py): the gradient against central finite
differences of L over head parameters; zero force weight reduces to the
energy-only gradient; a head with w2 = 0 leaves E and F unchanged.
"""
from __future__ import annotations

import numpy as np
import torch

from .model import atom_energies, _t
from .neighbors import wrap

_T = torch.float64
HEAD_KEYS = ("head_W1", "head_b1", "head_W2", "head_b2")


def pack(w: dict) -> np.ndarray:
    return np.concatenate([np.ravel(w[k]) for k in HEAD_KEYS])


def unpack(vec: np.ndarray, w: dict) -> dict:
    out = dict(w)
    o = 0
    for k in HEAD_KEYS:
        n = np.size(w[k])
        out[k] = np.asarray(vec[o:o + n]).reshape(np.shape(w[k]))
        o += n
    return out


def loss_and_grad(pos, species, box, edges, w, desc, n_layers, e_ref, f_ref, lam,
                  with_grad=True):
    """(L, dL/dtheta packed like ``pack``) for one snapshot."""
    box = np.asarray(box, dtype=np.float64)
    pos_t = torch.tensor(wrap(np.asarray(pos, dtype=np.float64), box), dtype=_T,
                         requires_grad=True)
    params = {k: torch.tensor(np.asarray(w[k], dtype=np.float64), requires_grad=with_grad)
              for k in HEAD_KEYS}
    wt = dict(w)
    wt.update(params)
    recv, send, code = edges
    Ei = atom_energies(pos_t, species, box, recv, send, code, wt, desc, n_layers, use_head=True)
    E = Ei.sum()
    (g,) = torch.autograd.grad(E, pos_t, create_graph=with_grad)
    F = -g
    N = pos.shape[0]
    L = ((E - float(e_ref)) / N) ** 2 + lam / (3.0 * N) * ((F - _t(f_ref)) ** 2).sum()
    if not with_grad:
        return float(L), None
    grads = torch.autograd.grad(L, [params[k] for k in HEAD_KEYS])
    return float(L.detach()), np.concatenate([gr.detach().numpy().ravel() for gr in grads])
