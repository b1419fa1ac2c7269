"""Electron sampler of the oracle (test infrastructure only).

Electron-sampler section: walkers start around their assigned nuclei and move
by Metropolis-Hastings on |psi|^2.  A proposal r' = r + s z (z standard normal,
all 3N coordinates of a walker at once) is accepted when log U <= A with
A = 2 log|psi(r')| - 2 log|psi(r)| and U uniform on (0, 1]; ties accept.
Random variates come from the counter streams of ``oracle.rng``.
"""
from __future__ import annotations

import numpy as np

from . import ansatz, ionic, rng


def init_walkers(nuclei, charges, n_up, n_down, partial_charges, n_walkers, seed, init_std,
                 dtype=np.float64, walker_offset: int = 0):
    """Algorithm 1 counts, spin split, then r = R_atom(e) + init_std * z."""
    n_el = n_up + n_down
    total_charge = int(round(float(np.sum(charges)))) - n_el
    counts = ionic.ionic_electron_counts([int(round(z)) for z in charges], partial_charges,
                                         total_charge)
    atoms = ionic.electron_atoms(counts, n_up, n_down)
    z = rng.walker_normals(seed, n_walkers, 3 * n_el, 0, rng.PURPOSE_INIT, walker_offset)
    return ionic.initial_positions(np.asarray(nuclei, np.float64), atoms, z, init_std, dtype), counts


def propose(r, seed: int, step: int, step_size: float, walker_offset: int = 0):
    """r' = r + step_size * z, computed in float64 and stored in the walker dtype."""
    B, N, _ = r.shape
    z = rng.walker_normals(seed, B, 3 * N, step, rng.PURPOSE_PROPOSAL, walker_offset)
    return (r.astype(np.float64) + z.reshape(B, N, 3) * float(step_size)).astype(r.dtype)


def metropolis(net, params, nuclei, r, log_psi, seed: int, n_steps: int, step_size: float,
               step_offset: int = 0, walker_offset: int = 0):
    """n_steps Metropolis steps; returns (r, log|psi|, accepted count per walker)."""
    r = np.array(r)
    lp = np.array(log_psi, dtype=np.float64)
    accepted = np.zeros(r.shape[0], dtype=np.int64)
    for s in range(n_steps):
        step = step_offset + s
        r_new = propose(r, seed, step, step_size, walker_offset)
        lp_new, _ = ansatz.log_psi(net, params, nuclei, r_new)
        log_u = rng.accept_log_uniform(seed, r.shape[0], step, walker_offset)
        acc = log_u <= 2.0 * (lp_new - lp)
        r = np.where(acc[:, None, None], r_new, r)
        lp = np.where(acc, lp_new, lp)
        accepted += acc
    return r, lp, accepted
