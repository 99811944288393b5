"""Layer diagnostics of the message-passing backbone (oracle; test
infrastructure only), as defined in Methods, "Mean Feature Shift and Linear
CKA":

  centred features   H~ = H - (1/N) 1 1^T H          (H: N nodes x d)
  MFS(i -> i+1)      = (1/N) || H~(i+1) - H~(i) ||_F
  CKA(i -> i+1)      = || H~(i)^T H~(i+1) ||_F^2
                       / ( || H~(i)^T H~(i) ||_F || H~(i+1)^T H~(i+1) ||_F )

Reading: the node feature matrix of a layer is the scalar (l = 0) feature
block h0 after that layer, d = F; layer 0 is the embedding.

Parity pins (tests/test_oracle_diagnostics.py): CKA(X, X) = 1 and CKA is
unchanged by an orthogonal rotation and an isotropic scaling of one side;
MFS(X, X) = 0 and MFS ignores a common shift of all nodes; a two-node
example worked by hand.
"""
from __future__ import annotations

import numpy as np

from .model import layer_features


def centre(h):
    h = np.asarray(h, dtype=np.float64)
    return h - h.mean(axis=0, keepdims=True)


def mfs(h_i, h_j) -> float:
    a, b = centre(h_i), centre(h_j)
    return float(np.linalg.norm(b - a) / a.shape[0])


def cka(h_i, h_j) -> float:
    a, b = centre(h_i), centre(h_j)
    num = np.linalg.norm(a.T @ b) ** 2
    return float(num / (np.linalg.norm(a.T @ a) * np.linalg.norm(b.T @ b)))


def layer_stats(pos, species, box, edges, w, desc, n_layers):
    """(MFS, CKA) arrays of length n_layers for the transitions i -> i + 1."""
    feats = layer_features(pos, species, box, edges, w, desc, n_layers)
    m = [mfs(feats[i], feats[i + 1]) for i in range(n_layers)]
    c = [cka(feats[i], feats[i + 1]) for i in range(n_layers)]
    return np.array(m), np.array(c)
