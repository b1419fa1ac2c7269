"""Pretraining loss of Eq. 5 (TEST INFRASTRUCTURE ONLY).

Eq. 5 compares the network's orbital matrices with Hartree-Fock orbitals at the sampled
electron positions: L = (1/N) sum_{k,i,j} (Phi_kij - Phi^HF_kij)^2, with k the determinant,
i the orbital and j the electron.  The text defines k, i and j but neither N nor the HF
variant; this module reads:

* Phi_kij = phi^k_i(r_j) for the electrons j of one spin, the orbital of Eq. 4 (projection
  times envelope, ``ansatz.orbital_matrices``); both spin blocks are summed;
* Phi^HF_kij = psi^HF_i(r_j), the i-th occupied orbital of that spin (in order of orbital
  energy) of the UHF calculation in STO-6G of ``oracle.scf``, the same for every k;
* N = the number of walkers of the batch (the sum also runs over them);
* the sign of each HF orbital makes its largest-magnitude coefficient positive; an occupied
  level that is degenerate has no unique orbitals and is refused.

Parity status: pinned by ``tests/test_oracle_pretrain.py`` (normalisation of the basis
functions by radial quadrature, the Roothaan-Hall equations, the HF energy recomputed from
the orbitals, antisymmetry of the HF determinants, and the variational identity: the mean
local energy of the HF determinant over |psi_HF|^2 equals the UHF energy).
"""
from __future__ import annotations

import numpy as np

from . import ansatz, rng, scf


def hf_state(nuclei, charges, n_up: int, n_down: int):
    """UHF in STO-6G: {basis, C_up [nbf, n_up], C_down [nbf, n_down], eps_up, eps_down, energy}."""
    nuclei = np.asarray(nuclei, np.float64)
    basis = scf.sto6g_basis(charges, nuclei)
    S, H, G, e_nn = scf.integrals(basis, nuclei, charges)
    e, Pa, Pb = scf.uhf(S, H, G, n_up, n_down, e_nn)
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T
    out = {"basis": basis, "energy": e, "S": S, "H": H, "G": G, "e_nn": e_nn}
    for name, P, n_occ in (("up", Pa, n_up), ("down", Pb, n_down)):
        J = np.einsum("pqrs,rs->pq", G, Pa + Pb)
        F = H + J - np.einsum("prqs,rs->pq", G, P)
        eps, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        if n_occ and n_occ < len(eps) and abs(eps[n_occ] - eps[n_occ - 1]) < 1e-8:
            raise ValueError("the highest occupied level is degenerate: the Eq. 5 target is not unique")
        if n_occ > 1 and np.min(np.diff(eps[:n_occ])) < 1e-8:
            raise ValueError("degenerate occupied orbitals: the Eq. 5 target is not unique")
        C = C[:, :n_occ].copy()
        for i in range(n_occ):
            k = int(np.argmax(np.abs(C[:, i])))
            if C[k, i] < 0:
                C[:, i] = -C[:, i]
        out[f"C_{name}"], out[f"eps_{name}"], out[f"F_{name}"] = C, eps[:n_occ], F
    return out


def _dims(f, r):
    d = r - f.centre
    return d, np.sum(d * d, -1)


def basis_values(basis, r):
    """chi_mu(r) for points r [..., 3] -> [..., nbf]."""
    r = np.asarray(r, np.float64)
    out = np.zeros(r.shape[:-1] + (len(basis),))
    for mu, f in enumerate(basis):
        d, r2 = _dims(f, r)
        poly = np.prod([d[..., a] ** f.lmn[a] for a in range(3)], axis=0)
        for a_k, c_k in zip(f.exps, f.coefs):
            out[..., mu] += c_k * scf.primitive_norm(a_k, f.lmn) * poly * np.exp(-a_k * r2)
    return out


def basis_laplacians(basis, r):
    """nabla^2 chi_mu(r): per direction, d^2/dx^2 of x^l e^(-a x^2) is
    l(l - 1) x^(l - 2) - 2a(2l + 1) x^l + 4a^2 x^(l + 2), times the other directions."""
    r = np.asarray(r, np.float64)
    out = np.zeros(r.shape[:-1] + (len(basis),))
    for mu, f in enumerate(basis):
        d, r2 = _dims(f, r)
        for a_k, c_k in zip(f.exps, f.coefs):
            g = c_k * scf.primitive_norm(a_k, f.lmn) * np.exp(-a_k * r2)
            for ax in range(3):
                l = f.lmn[ax]
                x = d[..., ax]
                d2 = -2 * a_k * (2 * l + 1) * x ** l + 4 * a_k * a_k * x ** (l + 2)
                if l >= 2:
                    d2 = d2 + l * (l - 1) * x ** (l - 2)
                other = np.prod([d[..., b] ** f.lmn[b] for b in range(3) if b != ax], axis=0)
                out[..., mu] += g * d2 * other
    return out


def hf_orbital_matrices(state, r):
    """Per spin [B, n_s, n_s]: element (i, j) = occupied HF orbital i at electron j of that spin."""
    r = np.asarray(r, np.float64)
    n_up = state["C_up"].shape[1]
    chi = basis_values(state["basis"], r)                      # [B, N, nbf]
    up = np.einsum("bjm,mi->bij", chi[:, :n_up], state["C_up"])
    down = np.einsum("bjm,mi->bij", chi[:, n_up:], state["C_down"])
    return up, down


def pretrain_loss_from(phis, hf_phis) -> float:
    """Eq. 5 from the network's matrices [B, K, n, n] per spin and the HF ones [B, n, n]."""
    B = phis[0].shape[0]
    tot = 0.0
    for A, H in zip(phis, hf_phis):
        tot += float(np.sum((A - H[:, None]) ** 2))
    return tot / B


def pretrain_loss(net, params, nuclei, r, state) -> float:
    return pretrain_loss_from(ansatz.orbital_matrices(net, params, nuclei, r), hf_orbital_matrices(state, r))


def hf_local_energy(state, nuclei, charges, r):
    """E_L of the HF determinant psi = det Phi_up det Phi_down (orbitals of one electron each,
    so nabla_j^2 det A / det A = sum_i (A^-1)_ji nabla^2 psi_i(r_j))."""
    r = np.asarray(r, np.float64)
    n_up = state["C_up"].shape[1]
    chi = basis_values(state["basis"], r)
    lap = basis_laplacians(state["basis"], r)
    kinetic = np.zeros(r.shape[0])
    for C, lo, hi in ((state["C_up"], 0, n_up), (state["C_down"], n_up, r.shape[1])):
        if hi == lo:
            continue
        A = np.einsum("bjm,mi->bij", chi[:, lo:hi], C)
        L = np.einsum("bjm,mi->bij", lap[:, lo:hi], C)
        Ainv = np.linalg.inv(A)
        kinetic += -0.5 * np.einsum("bij,bji->b", L, Ainv)
    v_ee, v_ne, v_nn = ansatz.potential_energy(np.asarray(nuclei, np.float64), np.asarray(charges, np.float64), r)
    return kinetic + v_ee + v_ne + v_nn


def hf_log_abs(state, r):
    up, down = hf_orbital_matrices(state, r)
    out = np.zeros(np.asarray(r).shape[0])
    for A in (up, down):
        if A.shape[1]:
            out += np.linalg.slogdet(A)[1]
    return out


def sample_hf(state, nuclei, charges, n_up, n_down, n_walkers, n_steps, step, seed):
    """Metropolis on |psi_HF|^2 with the oracle's streams (all-electron moves)."""
    from . import mcmc
    r, _ = mcmc.init_walkers(nuclei, charges, n_up, n_down, None, n_walkers, seed, 0.7)
    lp = hf_log_abs(state, r)
    for s in range(n_steps):
        prop = mcmc.propose(r, seed, s, step)
        lp_new = hf_log_abs(state, prop)
        acc = rng.accept_log_uniform(seed, n_walkers, s) <= 2.0 * (lp_new - lp)
        r = np.where(acc[:, None, None], prop, r)
        lp = np.where(acc, lp_new, lp)
    return r
