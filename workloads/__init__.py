"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module only *describes* inputs: nuclear geometries and charges, ansatz
sizes, walker counts and the Poisson job stream of the serving workload.  It
holds none of the method's arithmetic (no features, layers, determinants,
energies, random-number streams of the method or electron assignment), so the
oracle and the CUDA path can both import it without sharing any computation.

Geometries follow the systems named for the method's experiments: H2 at
1.4 bohr (Fig. 1 experiment), LiH at 3.015 bohr and its ions (Table 1
experiment, Algorithm 1), N2 at 2.068 bohr and CO at 2.132 bohr.  All lengths
are in bohr, energies in hartree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

ELEMENT_SYMBOLS = {1: "H", 2: "He", 3: "Li", 4: "Be", 5: "B", 6: "C", 7: "N", 8: "O",
                   9: "F", 10: "Ne", 11: "Na", 12: "Mg", 13: "Al", 14: "Si"}


@dataclass(frozen=True)
class Ansatz:
    """Sizes of the permutation-equivariant network (Sec. "FermiNet Model").

    n_layers: one-electron stream layers L (the two-electron stream has L-1).
    h1, h2: one- and two-electron feature widths.
    n_dets: determinants K.  envelope: "iso" (scalar sigma) or "aniso" (3x3 sigma, Eq. 4).
    """
    n_layers: int
    h1: int
    h2: int
    n_dets: int
    envelope: str = "iso"


@dataclass
class System:
    """Nuclei (bohr), nuclear charges Z, spin-resolved electron counts."""
    name: str
    nuclei: np.ndarray          # [M, 3] float64
    charges: np.ndarray         # [M] float64 (integer-valued Z)
    n_up: int
    n_down: int
    partial_charges: np.ndarray | None = None   # [M] Mulliken-style input of Algorithm 1

    @property
    def n_electrons(self) -> int:
        return self.n_up + self.n_down

    @property
    def total_charge(self) -> int:
        return int(round(float(self.charges.sum()))) - self.n_electrons


def _spins(n: int) -> Tuple[int, int]:
    return (n + 1) // 2, n // 2


def diatomic(name: str, z_a: int, z_b: int, bond: float, charge: int = 0,
             centered: bool = True, partial_charges=None) -> System:
    """Two nuclei on the z axis; centred at the origin or with atom A at the origin."""
    if centered:
        nuc = np.array([[0.0, 0.0, -bond / 2], [0.0, 0.0, bond / 2]])
    else:
        nuc = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, bond]])
    n = z_a + z_b - charge
    up, dn = _spins(n)
    pc = None if partial_charges is None else np.asarray(partial_charges, dtype=np.float64)
    return System(name, nuc, np.array([float(z_a), float(z_b)]), up, dn, pc)


def atom(z: int, charge: int = 0) -> System:
    n = z - charge
    up, dn = _spins(n)
    sym = ELEMENT_SYMBOLS[z] + {-1: "-", 0: "", 1: "+"}[charge]
    return System(sym, np.zeros((1, 3)), np.array([float(z)]), up, dn, None)


def h2(bond: float = 1.4) -> System:
    return diatomic("H2", 1, 1, bond)


def n2(bond: float = 2.068) -> System:
    return diatomic("N2", 7, 7, bond)


def co(bond: float = 2.132) -> System:
    return diatomic("CO", 6, 8, bond)


# Worked example of the ionic charge section: Mulliken partial charges of LiH+.
LIH_CATION_PARTIAL_CHARGES = (0.88694, 0.11306)


def lih(charge: int = 0, bond: float = 3.015) -> System:
    """LiH with Li at the origin and H at (0, 0, bond); cation 2 up/1 down, anion 3 up/2 down."""
    pc = LIH_CATION_PARTIAL_CHARGES if charge == 1 else None
    s = diatomic({-1: "LiH-", 0: "LiH", 1: "LiH+"}[charge], 3, 1, bond, charge=charge,
                 centered=False, partial_charges=pc)
    return s


def hydrogen_atom() -> System:
    return System("H", np.zeros((1, 3)), np.array([1.0]), 1, 0, None)


# --- the five workloads --------------------------------------------------------------

H2_SMALL = dict(system=h2, ansatz=Ansatz(2, 32, 8, 1, "iso"), walkers=256, mcmc_steps=20,
                step_size=0.02, init_std=1.0, seed=0, precision="fp64")
N2_LARGE = dict(system=n2, ansatz=Ansatz(4, 256, 32, 16, "aniso"), walkers=4096, mcmc_steps=10,
                step_size=0.02, init_std=1.0, seed=1, precision="fp32")
H2_PRECISION = dict(system=h2, ansatz=Ansatz(2, 32, 8, 1, "iso"), walkers=(4096, 16384),
                    mcmc_steps=20, step_size=0.02, init_std=1.0, seed=0, precision="bf16")
LIH_IONS = dict(system=lih, charges=(1, -1), ansatz=Ansatz(4, 128, 16, 8, "aniso"), walkers=4096,
                mcmc_steps=10, step_size=0.02, init_std=0.5, seed=4, precision="fp32")
SERVING_ANSATZ = Ansatz(4, 256, 32, 16, "aniso")


@dataclass
class Job:
    """One VMC energy request of the serving stream."""
    job_id: int
    arrival_s: float
    system: System
    n_walkers: int
    mcmc_steps: int = 50
    step_size: float = 0.02
    init_std: float = 1.0
    seed: int = 0


def serving_jobs(n_jobs: int = 1000, rate_per_s: float = 50.0, seed: int = 4,
                 min_walkers: int = 256, max_walkers: int = 4096,
                 mcmc_steps: int = 50) -> List[Job]:
    """Poisson job stream: half single atoms Z in 1..14 with charge -1/0/+1, half diatomics.

    Walker counts are log-uniform in [min_walkers, max_walkers].
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs: List[Job] = []
    molecules = [h2, lih, n2, co]
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        if rng.random() < 0.5:
            z = int(rng.integers(1, 15))
            q = int(rng.integers(-1, 2))
            sysm = atom(z, q)
        else:
            sysm = molecules[int(rng.integers(0, 4))]()
        nw = int(round(math.exp(rng.uniform(math.log(min_walkers), math.log(max_walkers)))))
        jobs.append(Job(i, t, sysm, nw, mcmc_steps, 0.02, 1.0, int(rng.integers(0, 2**31))))
    return jobs
