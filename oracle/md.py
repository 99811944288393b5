"""Velocity-Verlet NVE integration in FP64 (oracle; test infrastructure only).

The paper drives its potential with ASE molecular dynamics (Results, Table 2
conditions); the integrator here is the plain velocity-Verlet scheme:

  v <- v + dt/2 * kappa F / m
  r <- r + dt v                 then wrapped into the box
  F <- force(r)
  v <- v + dt/2 * kappa F / m

with kappa = 1 eV/(Angstrom amu) in Angstrom/fs^2.  The ledger records, per
step, the potential energy, the kinetic energy sum(m v^2) / (2 kappa) and
their sum.

Parity pins: on a harmonic oscillator the scheme's exact discrete solution
is known in closed form (tests/test_oracle_md.py); energy drift shrinks as
dt^2.
"""
from __future__ import annotations

import numpy as np

from synth import KAPPA
from .neighbors import wrap


def kinetic(vel, masses):
    return 0.5 * float((masses[:, None] * vel * vel).sum()) / KAPPA


def verlet(pos, vel, masses, box, force_fn, dt: float, n_steps: int, forces=None):
    """Integrate n_steps; force_fn(pos) -> (E, F).  Returns pos, vel, F, ledger
    [n_steps, 3] = (PE, KE, PE + KE) after each step."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    if forces is None:
        _, forces = force_fn(pos)
    ledger = np.zeros((n_steps, 3))
    acc = KAPPA * forces / masses[:, None]
    for s in range(n_steps):
        vel = vel + 0.5 * dt * acc
        pos = pos + dt * vel
        if box is not None:
            pos = wrap(pos, box)
        E, forces = force_fn(pos)
        acc = KAPPA * forces / masses[:, None]
        vel = vel + 0.5 * dt * acc
        ke = kinetic(vel, masses)
        ledger[s] = (E, ke, E + ke)
    return pos, vel, forces, ledger


def drift_mev_per_atom_ps(ledger, n_atoms: int, dt: float) -> float:
    """Least-squares slope of (E_tot(t) - E_tot(0)) / N in meV/atom/ps."""
    t = np.arange(1, ledger.shape[0] + 1) * dt * 1e-3      # ps
    y = (ledger[:, 2] - ledger[0, 2]) / n_atoms * 1e3     # meV/atom
    A = np.stack([t, np.ones_like(t)], 1)
    slope, _ = np.linalg.lstsq(A, y, rcond=None)[0]
    return float(slope)
