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

Langevin dynamics (the thermostat the paper's MD runs use, Results, Table 2
conditions) by the BAOAB splitting of Leimkuhler and Matthews (2013):

  v <- v + dt/2 * kappa F / m                       (B)
  r <- r + dt/2 v                                   (A)
  v <- c1 v + c2 sqrt(kB T kappa / m) xi            (O)  c1 = exp(-gamma dt),
  r <- r + dt/2 v, wrapped                          (A)  c2 = sqrt(1 - c1^2)
  F <- force(r);  v <- v + dt/2 * kappa F / m       (B)

xi: standard normals of the counter-based generator in synth (stream
STREAM_LANGEVIN, counter (step * N + atom) * 3 + axis), so every random
number the integrator draws is fixed by (seed, step, atom, axis).

Parity pins: on a harmonic oscillator the velocity-Verlet scheme's exact
discrete solution is known in closed form; energy drift shrinks as dt^2;
BAOAB with gamma = 0 is velocity Verlet; BAOAB samples the harmonic
oscillator's configurational distribution <k x^2> = kB T exactly
(tests/test_oracle_partition_md.py, tests/test_oracle_langevin.py).
"""
from __future__ import annotations

import math

import numpy as np

import synth
from synth import KAPPA, KB_EV
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


def langevin(pos, vel, masses, box, force_fn, dt: float, n_steps: int, T: float,
             gamma: float, seed: int, step0: int = 0, forces=None):
    """BAOAB Langevin steps (see the module docstring); step s of this call
    draws its noise with the counter of global step step0 + s.  Returns pos,
    vel, F, ledger [n_steps, 3] = (PE, KE, PE + KE) after each step."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    n = pos.shape[0]
    if forces is None:
        _, forces = force_fn(pos)
    c1 = math.exp(-gamma * dt)
    c2 = math.sqrt(1.0 - c1 * c1)
    sig = np.sqrt(KB_EV * T * KAPPA / masses)[:, None]
    ledger = np.zeros((n_steps, 3))
    idx = np.arange(3 * n, dtype=np.uint64).reshape(n, 3)
    for s in range(n_steps):
        vel = vel + 0.5 * dt * KAPPA * forces / masses[:, None]
        pos = pos + 0.5 * dt * vel
        xi = synth.normal_at(seed, synth.STREAM_LANGEVIN,
                             np.uint64((step0 + s) * 3 * n) + idx)
        vel = c1 * vel + c2 * sig * xi
        pos = pos + 0.5 * dt * vel
        if box is not None:
            pos = wrap(pos, box)
        E, forces = force_fn(pos)
        vel = vel + 0.5 * dt * KAPPA * forces / masses[:, None]
        ke = kinetic(vel, masses)
        ledger[s] = (E, ke, E + ke)
    return pos, vel, forces, ledger
