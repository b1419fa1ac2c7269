"""Ionic charge initialisation (Algorithm 1) and the spin split (test infrastructure only).

Algorithm 1 ("Charge Initialization Policy"): start from the neutral electron
counts (the atomic numbers) and the partial charges; while the ionic charge t
is non-zero, an anion (t < 0) gives one electron to the atom of lowest partial
charge and raises that partial charge by one, a cation (t > 0) takes one
electron from the atom of highest partial charge and lowers that partial charge
by one.  The loop runs |t| times.

Readings where the algorithm is silent (all stated, none printed by the method):
* ties in argmin/argmax go to the lowest atom index;
* an atom with no electron left is not eligible to lose one; if no atom is
  eligible the request is invalid (ValueError);
* without partial charges (no Hartree-Fock in this build) every atom gets t/M.

Spin split (the method is silent): per atom up = ceil(n/2), down = floor(n/2);
while the up total exceeds n_up, flip one up electron to down on the atom with
the largest (up - down), lowest index first; symmetric in the other direction.
Electrons are ordered up block then down block, each in atom order.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def ionic_electron_counts(atomic_numbers: Sequence[int], partial_charges: Sequence[float] | None,
                          total_charge: int) -> List[int]:
    """Algorithm 1: integer electrons per atom for an ion of charge ``total_charge``."""
    z = [int(v) for v in atomic_numbers]
    n_atoms = len(z)
    if partial_charges is None:
        charge = [total_charge / n_atoms] * n_atoms
    else:
        charge = [float(v) for v in partial_charges]
        if len(charge) != n_atoms:
            raise ValueError("one partial charge per atom is required")
    electron = list(z)
    t = int(total_charge)
    while t != 0:
        if t < 0:
            index = min(range(n_atoms), key=lambda a: (charge[a], a))
            electron[index] += 1
            t += 1
            charge[index] += 1
        else:
            eligible = [a for a in range(n_atoms) if electron[a] > 0]
            if not eligible:
                raise ValueError("cation charge exceeds the number of electrons")
            index = min(eligible, key=lambda a: (-charge[a], a))
            electron[index] -= 1
            t -= 1
            charge[index] -= 1
    return electron


def spin_split(counts: Sequence[int], n_up: int, n_down: int) -> Tuple[List[int], List[int]]:
    """Per-atom (up, down) counts with totals n_up and n_down."""
    if sum(counts) != n_up + n_down:
        raise ValueError("electron counts do not match n_up + n_down")
    up = [(c + 1) // 2 for c in counts]
    dn = [c // 2 for c in counts]
    while sum(up) > n_up:
        m = min((a for a in range(len(counts)) if up[a] > 0), key=lambda a: (-(up[a] - dn[a]), a))
        up[m] -= 1
        dn[m] += 1
    while sum(up) < n_up:
        m = min((a for a in range(len(counts)) if dn[a] > 0), key=lambda a: (-(dn[a] - up[a]), a))
        dn[m] -= 1
        up[m] += 1
    return up, dn


def electron_atoms(counts: Sequence[int], n_up: int, n_down: int) -> np.ndarray:
    """Atom index of every electron: up block then down block, each in atom order."""
    up, dn = spin_split(counts, n_up, n_down)
    order = [a for a in range(len(counts)) for _ in range(up[a])]
    order += [a for a in range(len(counts)) for _ in range(dn[a])]
    return np.array(order, dtype=np.int64)


def initial_positions(nuclei: np.ndarray, atoms_of_electrons: np.ndarray, normals: np.ndarray,
                      init_std: float, dtype=np.float64) -> np.ndarray:
    """r[w, e, :] = R[atom(e)] + init_std * z[w, 3e:3e+3] (product, then sum, both rounded)."""
    n_walkers = normals.shape[0]
    n_el = atoms_of_electrons.shape[0]
    z = normals.reshape(n_walkers, n_el, 3)
    centres = nuclei[atoms_of_electrons][None, :, :]
    r = centres + (z * float(init_std))
    return r.astype(dtype)
