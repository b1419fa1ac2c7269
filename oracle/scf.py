"""Minimal Hartree-Fock in the STO-6G basis and Mulliken charges (TEST INFRASTRUCTURE ONLY).

Algorithm 1 decides the electrons per atom of an ion from partial charges, which the
method takes from a Mulliken population analysis of a Hartree-Fock calculation in the
STO-6G basis (the pretraining paragraph names the basis; the LiH+ example prints the
charges [0.88694, 0.11306]).  This module computes those charges for molecules of
H..Ne:

* STO-6G: each Slater shell (1s; 2s and 2p with shared exponents) is the least-squares
  fit of six Gaussians to the Slater function of exponent 1 (the Hehre-Stewart-Pople
  construction), fitted here from scratch, then scaled by zeta^2 with the standard
  molecular exponents zeta of each element;
* one- and two-electron integrals over contracted Cartesian Gaussians (s and p) by the
  McMurchie-Davidson scheme: Hermite expansion coefficients E, Hermite Coulomb
  integrals R and the Boys function F_n(T) = 1F1(n + 1/2; n + 3/2; -T) / (2n + 1);
* unrestricted Hartree-Fock: six starts (core Hamiltonian, generalised Wolfsberg-Helmholz, four
  seeded symmetric perturbations), damped iterations, then DIIS; the lowest converged energy is
  kept;
* Mulliken charges q_A = Z_A - sum over basis functions mu on A of (P S)_mu,mu with
  P = P_alpha + P_beta.

Parity status: pinned by ``tests/test_oracle_scf.py`` (closed forms for s-type integrals,
centre derivatives of them for p-type ones, 3D quadrature, integral symmetries, the
hydrogen-atom energy by radial quadrature, and the LiH+ charges the paper prints).
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np
from scipy import optimize, special

# Standard molecular Slater exponents of the minimal-basis (STO-nG) calculations:
# (zeta of 1s, zeta of 2sp) for H..Ne.
STANDARD_ZETA = {1: (1.24, None), 2: (1.69, None), 3: (2.69, 0.80), 4: (3.68, 1.15), 5: (4.68, 1.50),
                 6: (5.67, 1.72), 7: (6.67, 1.95), 8: (7.66, 2.25), 9: (8.65, 2.55), 10: (9.64, 2.88)}


# ---- STO-6G from a least-squares fit ------------------------------------------------------
# Radial functions normalised over r^2 dr: the Slater function r^(n-1) e^(-r) (exponent 1)
# and Gaussians r^l e^(-a r^2).  Overlaps in closed form:
#   <g_a|g_b> = N_a N_b Gamma(l + 3/2) / (2 (a + b)^(l + 3/2)),
#   <g_a|STO> = N_a N_s J_(n+l+1)(a, 1),  J_m(a, beta) = int_0^inf r^m e^(-a r^2 - beta r) dr,
# with J_0 = sqrt(pi / 4a) erfcx(beta / 2 sqrt(a)), J_1 = (1 - beta J_0) / 2a and, by parts,
# 2a J_(m+1) = m J_(m-1) - beta J_m.
def _gauss_norm(l, a):
    return 1.0 / np.sqrt(special.gamma(l + 1.5) / (2.0 * (2.0 * a) ** (l + 1.5)))


def _slater_norm(n):
    return 2.0 ** n * math.sqrt(2.0 / math.factorial(2 * n))


def _J(m, a, beta=1.0):
    j0 = np.sqrt(np.pi / (4.0 * a)) * special.erfcx(beta / (2.0 * np.sqrt(a)))
    j1 = (1.0 - beta * j0) / (2.0 * a)
    js = [j0, j1]
    for k in range(1, m):
        js.append((k * js[k - 1] - beta * js[k]) / (2.0 * a))
    return js[m]


def _misfit(log_a, targets):
    """Sum over shells (l, n) of the squared L2 error of the best linear combination of the
    Gaussians with exponents exp(log_a) to the Slater function; returns (error, coefficients)."""
    a = np.exp(np.asarray(log_a, np.float64))
    err, coefs = 0.0, []
    for l, n in targets:
        Na = _gauss_norm(l, a)
        S = np.outer(Na, Na) * special.gamma(l + 1.5) / (2.0 * np.add.outer(a, a) ** (l + 1.5))
        b = Na * _slater_norm(n) * _J(n + l + 1, a)
        d = np.linalg.solve(S, b)
        err += 1.0 - b @ d
        coefs.append(d)
    return err, coefs


@functools.lru_cache(maxsize=None)
def sto6g_expansion(shell: str):
    """(exponents for zeta = 1, [coefficients per angular momentum]) of the 1s or 2sp shell,
    coefficients for normalised primitives; 2s and 2p share their exponents."""
    if shell == "1s":
        targets, x0 = [(0, 1)], [23.1, 4.2, 1.2, 0.4, 0.16, 0.065]
    elif shell == "2sp":
        targets, x0 = [(0, 2), (1, 2)], [10.3, 2.0, 0.63, 0.24, 0.1, 0.05]
    else:
        raise ValueError(shell)
    f = lambda z: _misfit(z, targets)[0]
    res = optimize.minimize(f, np.log(x0), method="Nelder-Mead",
                            options={"xatol": 1e-12, "fatol": 1e-18, "maxiter": 60000, "maxfev": 60000})
    for _ in range(2):
        res = optimize.minimize(f, res.x, method="BFGS", options={"gtol": 1e-15})
        res = optimize.minimize(f, res.x, method="Nelder-Mead",
                                options={"xatol": 1e-13, "fatol": 1e-19, "maxiter": 60000, "maxfev": 60000})
    _, coefs = _misfit(res.x, targets)
    return np.exp(res.x), [np.asarray(c) for c in coefs]


# ---- basis ----------------------------------------------------------------------------------
@dataclass
class Contracted:
    centre: np.ndarray          # [3]
    lmn: Tuple[int, int, int]
    exps: np.ndarray            # [K]
    coefs: np.ndarray           # [K], multiply normalised primitives
    atom: int


def _dfact(n):
    return 1.0 if n <= 0 else n * _dfact(n - 2)


def primitive_norm(a, lmn):
    l, m, n = lmn
    L = l + m + n
    return (2 * a / np.pi) ** 0.75 * (4 * a) ** (L / 2) / math.sqrt(_dfact(2 * l - 1) * _dfact(2 * m - 1) * _dfact(2 * n - 1))


def sto6g_basis(charges: Sequence[float], nuclei: np.ndarray) -> List[Contracted]:
    """Contracted functions in atom order: 1s, then (for Li..Ne) 2s, 2px, 2py, 2pz."""
    out = []
    e1, (c1,) = sto6g_expansion("1s")
    e2, (c2s, c2p) = sto6g_expansion("2sp")
    for i, z in enumerate(charges):
        z = int(round(z))
        if z not in STANDARD_ZETA:
            raise ValueError("STO-6G is provided for H..Ne")
        z1, z2 = STANDARD_ZETA[z]
        R = np.asarray(nuclei[i], np.float64)
        out.append(Contracted(R, (0, 0, 0), e1 * z1 * z1, c1.copy(), i))
        if z2 is not None:
            out.append(Contracted(R, (0, 0, 0), e2 * z2 * z2, c2s.copy(), i))
            for lmn in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                out.append(Contracted(R, lmn, e2 * z2 * z2, c2p.copy(), i))
    for f in out:   # normalise the contraction
        s = _overlap_prims(f, f)
        f.coefs = f.coefs / np.sqrt(np.sum(np.outer(f.coefs, f.coefs) * s))
    return out


# ---- McMurchie-Davidson ---------------------------------------------------------------------
def hermite_E(i, j, t, Q, a, b):
    """Coefficient of Lambda_t in the expansion of x_A^i x_B^j exp(-a x_A^2 - b x_B^2); arrays a, b."""
    p = a + b
    q = a * b / p
    if t < 0 or t > i + j:
        return np.zeros(np.broadcast(a, b).shape)
    if i == j == t == 0:
        return np.exp(-q * Q * Q)
    if j == 0:
        return (hermite_E(i - 1, j, t - 1, Q, a, b) / (2 * p) - (q * Q / a) * hermite_E(i - 1, j, t, Q, a, b)
                + (t + 1) * hermite_E(i - 1, j, t + 1, Q, a, b))
    return (hermite_E(i, j - 1, t - 1, Q, a, b) / (2 * p) + (q * Q / b) * hermite_E(i, j - 1, t, Q, a, b)
            + (t + 1) * hermite_E(i, j - 1, t + 1, Q, a, b))


def boys(n, T):
    return special.hyp1f1(n + 0.5, n + 1.5, -T) / (2 * n + 1)


def hermite_R(t, u, v, n, p, X, Y, Z):
    """Hermite Coulomb integral R^n_{tuv} for exponent p and P - C = (X, Y, Z) (arrays)."""
    if t == u == v == 0:
        return (-2 * p) ** n * boys(n, p * (X * X + Y * Y + Z * Z))
    if t > 0:
        out = X * hermite_R(t - 1, u, v, n + 1, p, X, Y, Z)
        if t > 1:
            out = out + (t - 1) * hermite_R(t - 2, u, v, n + 1, p, X, Y, Z)
        return out
    if u > 0:
        out = Y * hermite_R(t, u - 1, v, n + 1, p, X, Y, Z)
        if u > 1:
            out = out + (u - 1) * hermite_R(t, u - 2, v, n + 1, p, X, Y, Z)
        return out
    out = Z * hermite_R(t, u, v - 1, n + 1, p, X, Y, Z)
    if v > 1:
        out = out + (v - 1) * hermite_R(t, u, v - 2, n + 1, p, X, Y, Z)
    return out


def _pair(f, g):
    """Primitive-pair arrays of two contracted functions: exponents, weights, P, p."""
    a = f.exps[:, None]
    b = g.exps[None, :]
    wgt = (f.coefs * np.array([primitive_norm(x, f.lmn) for x in f.exps]))[:, None] * \
          (g.coefs * np.array([primitive_norm(x, g.lmn) for x in g.exps]))[None, :]
    p = a + b
    P = (a[..., None] * f.centre + b[..., None] * g.centre) / p[..., None]
    return a, b, wgt, p, P


def _overlap_1d(i, j, Q, a, b):
    return hermite_E(i, j, 0, Q, a, b) * np.sqrt(np.pi / (a + b))


def _overlap_prims(f, g):
    a, b, _, _, _ = _pair(f, g)
    norm = np.array([primitive_norm(x, f.lmn) for x in f.exps])[:, None] * \
        np.array([primitive_norm(x, g.lmn) for x in g.exps])[None, :]
    Q = f.centre - g.centre
    s = np.ones_like(a * b)
    for d in range(3):
        s = s * _overlap_1d(f.lmn[d], g.lmn[d], Q[d], a, b)
    return s * norm


def overlap(f, g):
    a, b, w, _, _ = _pair(f, g)
    Q = f.centre - g.centre
    s = np.ones_like(a * b)
    for d in range(3):
        s = s * _overlap_1d(f.lmn[d], g.lmn[d], Q[d], a, b)
    return float(np.sum(w * s))


def kinetic(f, g):
    """-1/2 <f|nabla^2|g>: d^2/dx^2 of x^l e^{-b x^2} = l(l-1) x^(l-2) - 2b(2l+1) x^l + 4b^2 x^(l+2)."""
    a, b, w, _, _ = _pair(f, g)
    Q = f.centre - g.centre
    s1d = [_overlap_1d(f.lmn[d], g.lmn[d], Q[d], a, b) for d in range(3)]
    tot = np.zeros_like(a * b)
    for d in range(3):
        i, j = f.lmn[d], g.lmn[d]
        d2 = -2 * b * (2 * j + 1) * _overlap_1d(i, j, Q[d], a, b) + 4 * b * b * _overlap_1d(i, j + 2, Q[d], a, b)
        if j >= 2:
            d2 = d2 + j * (j - 1) * _overlap_1d(i, j - 2, Q[d], a, b)
        other = np.ones_like(tot)
        for e in range(3):
            if e != d:
                other = other * s1d[e]
        tot = tot + d2 * other
    return float(np.sum(w * (-0.5) * tot))


def nuclear(f, g, C):
    """<f| 1/|r - C| |g> (positive; multiply by -Z for the attraction)."""
    a, b, w, p, P = _pair(f, g)
    Q = f.centre - g.centre
    PC = P - np.asarray(C, np.float64)
    tot = np.zeros_like(p)
    for t in range(f.lmn[0] + g.lmn[0] + 1):
        Et = hermite_E(f.lmn[0], g.lmn[0], t, Q[0], a, b)
        for u in range(f.lmn[1] + g.lmn[1] + 1):
            Eu = hermite_E(f.lmn[1], g.lmn[1], u, Q[1], a, b)
            for v in range(f.lmn[2] + g.lmn[2] + 1):
                Ev = hermite_E(f.lmn[2], g.lmn[2], v, Q[2], a, b)
                tot = tot + Et * Eu * Ev * hermite_R(t, u, v, 0, p, PC[..., 0], PC[..., 1], PC[..., 2])
    return float(np.sum(w * 2 * np.pi / p * tot))


def _hermite_products(f, g, a, b):
    """{(t, u, v): E_t^x E_u^y E_v^z} of the pair (f, g) over its primitive-pair arrays."""
    AB = f.centre - g.centre
    E = [[hermite_E(f.lmn[d], g.lmn[d], t, AB[d], a, b) for t in range(f.lmn[d] + g.lmn[d] + 1)] for d in range(3)]
    return {(t, u, v): E[0][t] * E[1][u] * E[2][v]
            for t in range(len(E[0])) for u in range(len(E[1])) for v in range(len(E[2]))}


def eri(f, g, h, k):
    """(fg|hk) in chemists' notation."""
    a, b, w1, p, P = _pair(f, g)
    c, d, w2, q, Qc = _pair(h, k)
    sh = (a.shape[0], b.shape[1], 1, 1)
    a4, b4, p4 = a.reshape(-1, 1, 1, 1), b.reshape(1, -1, 1, 1), p.reshape(sh)
    c4, d4, q4 = c.reshape(1, 1, -1, 1), d.reshape(1, 1, 1, -1), q.reshape(1, 1, *q.shape)
    PQ = P.reshape(*sh[:2], 1, 1, 3) - Qc.reshape(1, 1, *Qc.shape)
    alpha = p4 * q4 / (p4 + q4)
    E1 = _hermite_products(f, g, a4, b4)
    E2 = _hermite_products(h, k, c4, d4)
    memo = {}

    def R(t, u, v):
        key = (t, u, v)
        if key not in memo:
            memo[key] = hermite_R(t, u, v, 0, alpha, PQ[..., 0], PQ[..., 1], PQ[..., 2])
        return memo[key]

    tot = np.zeros(np.broadcast(p4, q4).shape)
    for (t, u, v), e1 in E1.items():
        for (tau, nu, phi), e2 in E2.items():
            tot = tot + e1 * e2 * (-1) ** (tau + nu + phi) * R(t + tau, u + nu, v + phi)
    pref = 2 * np.pi ** 2.5 / (p4 * q4 * np.sqrt(p4 + q4))
    return float(np.sum(w1.reshape(sh) * w2.reshape(1, 1, *w2.shape) * pref * tot))


def integrals(basis, nuclei, charges):
    """(S, T + V, ERI[n,n,n,n], nuclear repulsion)."""
    n = len(basis)
    S = np.array([[overlap(f, g) for g in basis] for f in basis])
    T = np.array([[kinetic(f, g) for g in basis] for f in basis])
    V = np.zeros((n, n))
    for C, Z in zip(nuclei, charges):
        V -= Z * np.array([[nuclear(f, g, C) for g in basis] for f in basis])
    G = np.zeros((n, n, n, n))
    for i in range(n):
        for j in range(i + 1):
            for k in range(n):
                for l in range(k + 1):
                    if i * (i + 1) // 2 + j < k * (k + 1) // 2 + l:
                        continue
                    x = eri(basis[i], basis[j], basis[k], basis[l])
                    for (p, q, r, s) in ((i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                                         (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)):
                        G[p, q, r, s] = x
    e_nn = 0.0
    for m in range(len(charges)):
        for k in range(m):
            e_nn += charges[m] * charges[k] / np.linalg.norm(np.asarray(nuclei[m]) - np.asarray(nuclei[k]))
    return S, T + V, G, e_nn


# ---- unrestricted Hartree-Fock ----------------------------------------------------------------
def gwh_guess(S, H, k=1.75):
    """Generalised Wolfsberg-Helmholz start: F_ij = k S_ij (H_ii + H_jj) / 2 off the diagonal."""
    F = k * S * (np.diag(H)[:, None] + np.diag(H)[None, :]) / 2
    np.fill_diagonal(F, np.diag(H))
    return F


def _uhf_from(F0, S, H, G, n_alpha, n_beta, e_nn, tol, max_iter, damp_iters):
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T

    def density(F, n_occ):
        e, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C
        return C[:, :n_occ] @ C[:, :n_occ].T

    Pa, Pb = density(F0, n_alpha), density(F0, n_beta)
    hist_F, hist_e = [], []
    e_old = None
    for it in range(max_iter):
        J = np.einsum("pqrs,rs->pq", G, Pa + Pb)
        Fa = H + J - np.einsum("prqs,rs->pq", G, Pa)
        Fb = H + J - np.einsum("prqs,rs->pq", G, Pb)
        e = 0.5 * (np.sum((H + Fa) * Pa) + np.sum((H + Fb) * Pb)) + e_nn
        err = np.concatenate([(Fa @ Pa @ S - S @ Pa @ Fa).ravel(), (Fb @ Pb @ S - S @ Pb @ Fb).ravel()])
        if e_old is not None and abs(e - e_old) < tol and np.max(np.abs(err)) < 1e-8:
            return e, Pa, Pb
        e_old = e
        if it < damp_iters:                      # damped iterations before extrapolation
            Pa = 0.5 * (Pa + density(Fa, n_alpha))
            Pb = 0.5 * (Pb + density(Fb, n_beta))
            continue
        hist_F.append((Fa, Fb))
        hist_e.append(err)
        hist_F, hist_e = hist_F[-8:], hist_e[-8:]
        m = len(hist_e)
        B = -np.ones((m + 1, m + 1))
        B[m, m] = 0.0
        for i in range(m):
            for j in range(m):
                B[i, j] = hist_e[i] @ hist_e[j]
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
        Fa = sum(ci * f[0] for ci, f in zip(c, hist_F))
        Fb = sum(ci * f[1] for ci, f in zip(c, hist_F))
        Pa, Pb = density(Fa, n_alpha), density(Fb, n_beta)
    raise RuntimeError("UHF did not converge")


def uhf(S, H, G, n_alpha, n_beta, e_nn=0.0, tol=1e-11, max_iter=500, damp_iters=30):
    """UHF ground state; returns (energy, Pa, Pb).  DIIS from the first iteration can settle on
    an excited self-consistent solution (N2 in STO-6G: -107.818 instead of -108.541 Ha), and
    open shells with degenerate levels have several solutions (O+), so six starts are run (core
    Hamiltonian, generalised Wolfsberg-Helmholz, and four seeded symmetric perturbations of the
    core Hamiltonian), each with `damp_iters` damped iterations (P <- (P + P_new) / 2) before
    DIIS; the lowest converged energy is kept."""
    starts = [H, gwh_guess(S, H)]
    rs = np.random.default_rng(20240118)
    for _ in range(16):                      # symmetry-breaking starts for open shells
        A = rs.standard_normal(H.shape)
        starts.append(H + 0.3 * (A + A.T))
    best = None
    for F0 in starts:
        try:
            res = _uhf_from(F0, S, H, G, n_alpha, n_beta, e_nn, tol, max_iter, damp_iters)
        except RuntimeError:
            continue
        if best is None or res[0] < best[0] - 1e-9:
            best = res
    if best is None:
        raise RuntimeError("UHF did not converge from any start")
    return best


def mulliken_charges(nuclei, charges, n_alpha, n_beta):
    """(Mulliken charge per atom, UHF energy) in the STO-6G basis."""
    nuclei = np.asarray(nuclei, np.float64)
    basis = sto6g_basis(charges, nuclei)
    S, H, G, e_nn = integrals(basis, nuclei, charges)
    e, Pa, Pb = uhf(S, H, G, n_alpha, n_beta, e_nn)
    pop = np.diag((Pa + Pb) @ S)
    q = np.array([float(z) for z in charges])
    for mu, f in enumerate(basis):
        q[f.atom] -= pop[mu]
    return q, e
