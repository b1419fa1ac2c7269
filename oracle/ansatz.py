"""FP64 wavefunction, forward-Laplacian local energy and potentials (test infrastructure only).

What is computed (method sections "FermiNet Model", Eqs. 2-4):

* features: one-electron stream input h0_i = [r_i - R_m, |r_i - R_m|] for every
  nucleus m (4M values); two-electron stream input g0_ij = [r_i - r_j, |r_i - r_j|]
  (the diagonal pair is identically zero with zero derivatives).
* layers (reading of the stream description after the cited FermiNet design):
  f_i = [h_i, mean_{j up} h_j, mean_{j down} h_j, mean_{j up} g_ij, mean_{j down} g_ij]
  h_i <- tanh(V f_i + b) (+ h_i for layers l >= 1),
  g_ij <- tanh(W g_ij + c) (+ g_ij for pair layers l >= 1), L-1 pair layers.
  A mean over an empty spin group is zero.
* orbitals (Eq. 4): phi^{k,a}_i(r_j) = (w^{k,a}_i . h^L_j + g^{k,a}_i)
  * sum_m pi^{k,a}_{i,m} exp(-|sigma^{k,a}_{i,m} (r_j - R_m)|), with sigma a 3x3
  matrix ("aniso") or a scalar multiplying |r_j - R_m| ("iso").
* psi = sum_k det[phi^{k,up}] det[phi^{k,down}] (an empty spin block has
  determinant 1); log|psi| by a signed log-sum-exp.
* kinetic energy (Eq. 3, read as the sum over all 3N coordinates):
  -1/2 sum_c [(d log|psi| / d x_c)^2 + d^2 log|psi| / d x_c^2].
* potentials (Eq. 2 terms): V_ee = sum_{i<j} 1/r_ij, V_ne = -sum_{i,m} Z_m/|r_i-R_m|,
  V_nn = sum_{m<n} Z_m Z_n/|R_m - R_n|.

The exact Laplacian is obtained by carrying, through every operation, the
value, the gradient with respect to all 3N electron coordinates and the
Laplacian (a "jet"); this is the plain chain and product rule, written per
operation.  ``fd_log_psi_derivatives`` is an independent central-difference
path used to pin it.

Parameter blob (one flat array, in this order):
  for layer l = 0..L-1: V_l [h1, 3 d_h + 2 d_g], b_l [h1],
      and for l < L-1: W_l [h2, d_g], c_l [h2]
      (d_h = 4M, d_g = 4 at l = 0; d_h = h1, d_g = h2 after);
  for spin a in (up, down) with n_a > 0: w_a [K n_a, h1], g_a [K n_a];
  for spin a in (up, down) with n_a > 0: pi_a [K n_a, M],
      sigma_a [K n_a, M] (iso) or [K n_a, M, 3, 3] (aniso).
Orbital rows are ordered (k, i): row = k * n_a + i.
Initialisation: dense weights and biases ~ N(0,1)/sqrt(fan_in) from the
parameter stream of ``rng``; pi = 1 and sigma = 1 (identity for aniso).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

from . import rng


@dataclass(frozen=True)
class Net:
    n_nuclei: int
    n_up: int
    n_down: int
    n_layers: int
    h1: int
    h2: int
    n_dets: int
    envelope: str = "iso"

    @property
    def n_el(self) -> int:
        return self.n_up + self.n_down


def param_layout(net: Net) -> List[Tuple[str, Tuple[int, ...], int, str]]:
    """(name, shape, fan_in, init kind) in blob order."""
    M, L, h1, h2, K = net.n_nuclei, net.n_layers, net.h1, net.h2, net.n_dets
    out = []
    for l in range(L):
        d_h = 4 * M if l == 0 else h1
        d_g = 4 if l == 0 else h2
        f_in = 3 * d_h + 2 * d_g
        out.append((f"V{l}", (h1, f_in), f_in, "normal"))
        out.append((f"b{l}", (h1,), f_in, "normal"))
        if l < L - 1:
            out.append((f"W{l}", (h2, d_g), d_g, "normal"))
            out.append((f"c{l}", (h2,), d_g, "normal"))
    for a, n_a in (("up", net.n_up), ("down", net.n_down)):
        if n_a:
            out.append((f"w_{a}", (K * n_a, h1), h1, "normal"))
            out.append((f"g_{a}", (K * n_a,), h1, "normal"))
    for a, n_a in (("up", net.n_up), ("down", net.n_down)):
        if n_a:
            out.append((f"pi_{a}", (K * n_a, M), 1, "one"))
            if net.envelope == "iso":
                out.append((f"sigma_{a}", (K * n_a, M), 1, "one"))
            else:
                out.append((f"sigma_{a}", (K * n_a, M, 3, 3), 1, "identity"))
    return out


def param_count(net: Net) -> int:
    return int(sum(int(np.prod(s)) for _, s, _, _ in param_layout(net)))


def unpack(net: Net, blob: np.ndarray) -> Dict[str, np.ndarray]:
    blob = np.asarray(blob)
    out, off = {}, 0
    for name, shape, _, _ in param_layout(net):
        n = int(np.prod(shape))
        out[name] = blob[off:off + n].reshape(shape)
        off += n
    if off != blob.shape[0]:
        raise ValueError(f"parameter blob has {blob.shape[0]} values, layout needs {off}")
    return out


def init_params(net: Net, seed: int) -> np.ndarray:
    """Blob of float64 initial parameters (normal draws times 1/sqrt(fan_in))."""
    blob = np.empty(param_count(net), dtype=np.float64)
    off = 0
    for _, shape, fan_in, kind in param_layout(net):
        n = int(np.prod(shape))
        if kind == "normal":
            j = np.arange(off, off + n, dtype=np.uint64)
            z = rng.normals(seed, np.uint64(0), np.uint64(0), np.uint64(rng.PURPOSE_PARAMS), j)
            blob[off:off + n] = z * (1.0 / np.sqrt(float(fan_in)))
        elif kind == "one":
            blob[off:off + n] = 1.0
        else:
            blob[off:off + n] = np.broadcast_to(np.eye(3), shape).reshape(-1)
        off += n
    return blob


# ----------------------------------------------------------------------------------------
# determinants: LU with partial pivoting (first maximal |pivot| in row order)
# ----------------------------------------------------------------------------------------

def lu_factor(a: np.ndarray):
    """Doolittle LU with partial pivoting over the last two axes.

    Returns (lu, perm, perm_sign): rows of ``a`` taken in order ``perm`` equal L U,
    with the unit lower factor stored below the diagonal of ``lu``.
    """
    shape = a.shape
    n = shape[-1]
    lu = np.array(a, dtype=np.float64).reshape(-1, n, n)
    p = lu.shape[0]
    ar = np.arange(p)
    perm = np.tile(np.arange(n), (p, 1))
    sign = np.ones(p)
    for c in range(n):
        piv = c + np.argmax(np.abs(lu[:, c:, c]), axis=1)
        swap = piv != c
        row_c = lu[ar, c].copy()
        row_p = lu[ar, piv].copy()
        lu[ar, c] = row_p
        lu[ar, piv] = row_c
        pc = perm[ar, c].copy()
        perm[ar, c] = perm[ar, piv]
        perm[ar, piv] = pc
        sign = np.where(swap, -sign, sign)
        if c + 1 < n:
            factor = lu[:, c + 1:, c] / lu[:, c, c][:, None]
            lu[:, c + 1:, c] = factor
            lu[:, c + 1:, c + 1:] -= factor[:, :, None] * lu[:, c, None, c + 1:]
    return lu.reshape(shape), perm.reshape(shape[:-1]), sign.reshape(shape[:-2])


def slogdet(a: np.ndarray):
    """(sign, log|det|) from the LU factors; an empty matrix has determinant 1."""
    n = a.shape[-1]
    if n == 0:
        return np.ones(a.shape[:-2]), np.zeros(a.shape[:-2])
    lu, _, psign = lu_factor(a)
    diag = np.diagonal(lu, axis1=-2, axis2=-1)
    return psign * np.prod(np.sign(diag), axis=-1), np.sum(np.log(np.abs(diag)), axis=-1)


def inverse(a: np.ndarray) -> np.ndarray:
    """A^{-1} by forward and back substitution on the pivoted LU factors."""
    n = a.shape[-1]
    lu, perm, _ = lu_factor(a)
    lu = lu.reshape(-1, n, n)
    perm = perm.reshape(-1, n)
    p = lu.shape[0]
    # right-hand side: rows of the identity in pivot order
    y = np.zeros((p, n, n))
    y[np.arange(p)[:, None], np.arange(n)[None, :], perm] = 1.0
    for i in range(n):                      # L y = P I (unit diagonal)
        for k in range(i):
            y[:, i, :] -= lu[:, i, k, None] * y[:, k, :]
    x = y
    for i in range(n - 1, -1, -1):          # U x = y
        for k in range(i + 1, n):
            x[:, i, :] -= lu[:, i, k, None] * x[:, k, :]
        x[:, i, :] /= lu[:, i, i, None]
    return x.reshape(a.shape)


# ----------------------------------------------------------------------------------------
# value-only wavefunction
# ----------------------------------------------------------------------------------------

def _spin_mean(x: np.ndarray, axis: int, lo: int, hi: int) -> np.ndarray:
    if hi == lo:
        shape = list(x.shape)
        del shape[axis]
        return np.zeros(shape, dtype=x.dtype)
    return np.take(x, np.arange(lo, hi), axis=axis).mean(axis=axis)


def _envelope_value(net: Net, p: Dict[str, np.ndarray], a: str, d: np.ndarray) -> np.ndarray:
    """sum_m pi exp(-|sigma d_m|) for d [B, n_a, M, 3] -> [B, n_a, K n_a]."""
    pi = p[f"pi_{a}"]                       # [KO, M]
    sig = p[f"sigma_{a}"]
    if net.envelope == "iso":
        dist = np.sqrt(np.sum(d * d, axis=-1))                      # [B, j, M]
        s = sig[None, None, :, :] * dist[:, :, None, :]             # [B, j, KO, M]
    else:
        u = np.einsum("omxy,bjmy->bjomx", sig, d)                   # [B, j, KO, M, 3]
        s = np.sqrt(np.sum(u * u, axis=-1))
    return np.sum(pi[None, None] * np.exp(-s), axis=-1)


def orbital_matrices(net: Net, params: np.ndarray, nuclei: np.ndarray, r: np.ndarray):
    """Per spin: A[b, k, i, j] = phi^{k}_i(r_j) for the electrons j of that spin."""
    p = unpack(net, params)
    h, _ = _streams(net, p, nuclei, r)
    mats = []
    for a, lo, hi in (("up", 0, net.n_up), ("down", net.n_up, net.n_el)):
        n_a = hi - lo
        if n_a == 0:
            mats.append(np.zeros((r.shape[0], net.n_dets, 0, 0)))
            continue
        proj = h[:, lo:hi] @ p[f"w_{a}"].T + p[f"g_{a}"]             # [B, j, KO]
        d = r[:, lo:hi, None, :] - nuclei[None, None]                 # [B, j, M, 3]
        phi = proj * _envelope_value(net, p, a, d)
        mats.append(phi.reshape(r.shape[0], n_a, net.n_dets, n_a).transpose(0, 2, 3, 1))
    return mats


def _streams(net: Net, p, nuclei, r):
    r = np.asarray(r, dtype=np.float64)
    B, N, _ = r.shape
    d_en = r[:, :, None, :] - nuclei[None, None]
    h = np.concatenate([d_en, np.sqrt(np.sum(d_en * d_en, -1))[..., None]], -1).reshape(B, N, -1)
    d_ee = r[:, :, None, :] - r[:, None, :, :]
    g = np.concatenate([d_ee, np.sqrt(np.sum(d_ee * d_ee, -1))[..., None]], -1)
    nu = net.n_up
    for l in range(net.n_layers):
        hu = _spin_mean(h, 1, 0, nu)[:, None, :].repeat(N, 1)
        hd = _spin_mean(h, 1, nu, N)[:, None, :].repeat(N, 1)
        gu = _spin_mean(g, 2, 0, nu)
        gd = _spin_mean(g, 2, nu, N)
        f = np.concatenate([h, hu, hd, gu, gd], -1)
        h_new = np.tanh(f @ p[f"V{l}"].T + p[f"b{l}"])
        if l > 0:
            h_new = h_new + h
        if l < net.n_layers - 1:
            g_new = np.tanh(g @ p[f"W{l}"].T + p[f"c{l}"])
            if l > 0:
                g_new = g_new + g
            g = g_new
        h = h_new
    return h, g


def combine_dets(sign_k: np.ndarray, logdet_k: np.ndarray):
    """log|sum_k s_k exp(l_k)| and its sign, plus the weights rho_k = D_k / psi."""
    m = np.max(logdet_k, axis=-1, keepdims=True)
    w = sign_k * np.exp(logdet_k - m)
    s = np.sum(w, axis=-1)
    return np.sign(s), m[..., 0] + np.log(np.abs(s)), w / s[..., None]


def log_psi(net: Net, params: np.ndarray, nuclei: np.ndarray, r: np.ndarray):
    """(log|psi|, sign psi) per walker, value only."""
    a_up, a_dn = orbital_matrices(net, params, nuclei, r)
    s_up, l_up = slogdet(a_up)
    s_dn, l_dn = slogdet(a_dn)
    sign, lp, _ = combine_dets(s_up * s_dn, l_up + l_dn)
    return lp, sign


# ----------------------------------------------------------------------------------------
# forward-Laplacian jets: value v [..., C], gradient g [..., 3N, C], Laplacian l [..., C]
# ----------------------------------------------------------------------------------------

@dataclass
class Jet:
    v: np.ndarray
    g: np.ndarray
    l: np.ndarray


def _jet_linear(x: Jet, w: np.ndarray, b: np.ndarray | None = None) -> Jet:
    v = x.v @ w.T
    if b is not None:
        v = v + b
    return Jet(v, x.g @ w.T, x.l @ w.T)


def _jet_tanh(x: Jet) -> Jet:
    h = np.tanh(x.v)
    d = 1.0 - h * h
    return Jet(h, d[..., None, :] * x.g, d * x.l - 2.0 * h * d * np.sum(x.g * x.g, axis=-2))


def _jet_add(a: Jet, b: Jet) -> Jet:
    return Jet(a.v + b.v, a.g + b.g, a.l + b.l)


def _jet_cat(parts: List[Jet]) -> Jet:
    return Jet(np.concatenate([q.v for q in parts], -1), np.concatenate([q.g for q in parts], -1),
               np.concatenate([q.l for q in parts], -1))


def _jet_spin_mean(x: Jet, axis: int, lo: int, hi: int) -> Jet:
    return Jet(_spin_mean(x.v, axis, lo, hi), _spin_mean(x.g, axis, lo, hi),
               _spin_mean(x.l, axis, lo, hi))


def _jet_expand(x: Jet, n: int) -> Jet:
    return Jet(x.v[:, None].repeat(n, 1), x.g[:, None].repeat(n, 1), x.l[:, None].repeat(n, 1))


def _jet_mul(a: Jet, b: Jet) -> Jet:
    v = a.v * b.v
    g = a.g * b.v[..., None, :] + a.v[..., None, :] * b.g
    l = a.l * b.v + a.v * b.l + 2.0 * np.sum(a.g * b.g, axis=-2)
    return Jet(v, g, l)


def feature_jets(nuclei: np.ndarray, r: np.ndarray) -> Tuple[Jet, Jet]:
    """Input features with their exact gradients and Laplacians."""
    B, N, _ = r.shape
    M = nuclei.shape[0]
    T = 3 * N
    d_en = r[:, :, None, :] - nuclei[None, None]                      # [B, N, M, 3]
    dist = np.sqrt(np.sum(d_en * d_en, -1))                          # [B, N, M]
    hv = np.concatenate([d_en, dist[..., None]], -1).reshape(B, N, 4 * M)
    hg = np.zeros((B, N, T, 4 * M))
    hl = np.zeros((B, N, 4 * M))
    for i in range(N):
        for m in range(M):
            for c in range(3):
                hg[:, i, 3 * i + c, 4 * m + c] = 1.0
                hg[:, i, 3 * i + c, 4 * m + 3] = d_en[:, i, m, c] / dist[:, i, m]
            hl[:, i, 4 * m + 3] = 2.0 / dist[:, i, m]
    d_ee = r[:, :, None, :] - r[:, None, :, :]                        # [B, N, N, 3]
    dee = np.sqrt(np.sum(d_ee * d_ee, -1))
    gv = np.concatenate([d_ee, dee[..., None]], -1)
    gg = np.zeros((B, N, N, T, 4))
    gl = np.zeros((B, N, N, 4))
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            for c in range(3):
                gg[:, i, j, 3 * i + c, c] = 1.0
                gg[:, i, j, 3 * j + c, c] = -1.0
                unit = d_ee[:, i, j, c] / dee[:, i, j]
                gg[:, i, j, 3 * i + c, 3] = unit
                gg[:, i, j, 3 * j + c, 3] = -unit
            gl[:, i, j, 3] = 4.0 / dee[:, i, j]
    return Jet(hv, hg, hl), Jet(gv, gg, gl)


def _envelope_jet(net: Net, p, a: str, nuclei, r: np.ndarray, lo: int, hi: int) -> Jet:
    """Envelope of the electrons lo..hi-1 of spin a; derivatives only along their own coordinates."""
    B, N, _ = r.shape
    n_a = hi - lo
    pi = p[f"pi_{a}"]
    sig = p[f"sigma_{a}"]
    d = r[:, lo:hi, None, :] - nuclei[None, None]                       # [B, j, M, 3]
    if net.envelope == "iso":
        dist = np.sqrt(np.sum(d * d, -1))                               # [B, j, M]
        s = sig[None, None] * dist[:, :, None, :]                       # [B, j, KO, M]
        grad_s = sig[None, None, :, :, None] * (d / dist[..., None])[:, :, None, :, :]
        lap_s = 2.0 * sig[None, None] / dist[:, :, None, :]
    else:
        u = np.einsum("omxy,bjmy->bjomx", sig, d)                       # [B, j, KO, M, 3]
        s = np.sqrt(np.sum(u * u, -1))                                  # [B, j, KO, M]
        stu = np.einsum("omxy,bjomx->bjomy", sig, u)                    # sigma^T u
        grad_s = stu / s[..., None]
        frob = np.sum(sig * sig, axis=(-1, -2))                         # [KO, M]
        lap_s = (frob[None, None] - np.sum(stu * stu, -1) / (s * s)) / s
    e = pi[None, None] * np.exp(-s)                                     # [B, j, KO, M]
    v = e.sum(-1)
    grad = -np.sum(e[..., None] * grad_s, axis=-2)                      # [B, j, KO, 3]
    lap = np.sum(e * (np.sum(grad_s * grad_s, -1) - lap_s), axis=-1)    # [B, j, KO]
    g = np.zeros((B, n_a, 3 * N, v.shape[-1]))
    for jj in range(n_a):
        for c in range(3):
            g[:, jj, 3 * (lo + jj) + c, :] = grad[:, jj, :, c]
    return Jet(v, g, lap)


def _logdet_jet(a: Jet):
    """sign, log|det A|, its gradient over all coordinates and its Laplacian.

    d log|det A| = tr(A^-1 dA);  Laplacian = tr(A^-1 lap A) - sum_t tr((A^-1 d_t A)^2).
    a.v [B, K, n, n]; a.g [B, K, n, n, T]; a.l [B, K, n, n].
    """
    B, K, n, _ = a.v.shape
    T = a.g.shape[-1]
    if n == 0:
        return np.ones((B, K)), np.zeros((B, K)), np.zeros((B, K, T)), np.zeros((B, K))
    sign, ld = slogdet(a.v)
    ainv = inverse(a.v)
    grad = np.einsum("bkji,bkijt->bkt", ainv, a.g)
    prod = np.einsum("bkij,bkjlt->bkilt", ainv, a.g)
    tr2 = np.einsum("bkilt,bklit->bkt", prod, prod)
    lap = np.einsum("bkji,bkij->bk", ainv, a.l) - np.sum(tr2, -1)
    return sign, ld, grad, lap


def log_psi_derivatives(net: Net, params: np.ndarray, nuclei: np.ndarray, r: np.ndarray):
    """log|psi|, sign, gradient [B, 3N] and Laplacian [B] of log|psi| via jets."""
    p = unpack(net, params)
    r = np.asarray(r, dtype=np.float64)
    B, N, _ = r.shape
    nu = net.n_up
    h, g = feature_jets(nuclei, r)
    for l in range(net.n_layers):
        hu = _jet_expand(_jet_spin_mean(h, 1, 0, nu), N)
        hd = _jet_expand(_jet_spin_mean(h, 1, nu, N), N)
        gu = _jet_spin_mean(g, 2, 0, nu)
        gd = _jet_spin_mean(g, 2, nu, N)
        f = _jet_cat([h, hu, hd, gu, gd])
        h_new = _jet_tanh(_jet_linear(f, p[f"V{l}"], p[f"b{l}"]))
        if l > 0:
            h_new = _jet_add(h_new, h)
        if l < net.n_layers - 1:
            g_new = _jet_tanh(_jet_linear(g, p[f"W{l}"], p[f"c{l}"]))
            if l > 0:
                g_new = _jet_add(g_new, g)
            g = g_new
        h = h_new
    sign_k = np.ones((B, net.n_dets))
    ld_k = np.zeros((B, net.n_dets))
    grad_k = np.zeros((B, net.n_dets, 3 * N))
    lap_k = np.zeros((B, net.n_dets))
    for a, lo, hi in (("up", 0, nu), ("down", nu, N)):
        n_a = hi - lo
        if n_a == 0:
            continue
        hj = Jet(h.v[:, lo:hi], h.g[:, lo:hi], h.l[:, lo:hi])
        proj = _jet_linear(hj, p[f"w_{a}"], p[f"g_{a}"])                  # [B, j, KO]
        phi = _jet_mul(proj, _envelope_jet(net, p, a, nuclei, r, lo, hi))
        K = net.n_dets
        av = phi.v.reshape(B, n_a, K, n_a).transpose(0, 2, 3, 1)
        ag = phi.g.reshape(B, n_a, 3 * N, K, n_a).transpose(0, 3, 4, 1, 2)
        al = phi.l.reshape(B, n_a, K, n_a).transpose(0, 2, 3, 1)
        s, ld, gr, lp = _logdet_jet(Jet(av, ag, al))
        sign_k *= s
        ld_k += ld
        grad_k += gr
        lap_k += lp
    sign, lpsi, rho = combine_dets(sign_k, ld_k)
    grad = np.einsum("bk,bkt->bt", rho, grad_k)
    lap = np.einsum("bk,bk->b", rho, lap_k + np.sum(grad_k * grad_k, -1)) - np.sum(grad * grad, -1)
    return lpsi, sign, grad, lap


def potential_energy(nuclei: np.ndarray, charges: np.ndarray, r: np.ndarray):
    """(V_ee, V_ne, V_nn) per walker."""
    r = np.asarray(r, dtype=np.float64)
    B, N, _ = r.shape
    M = nuclei.shape[0]
    v_ee = np.zeros(B)
    for i in range(N):
        for j in range(i + 1, N):
            v_ee += 1.0 / np.sqrt(np.sum((r[:, i] - r[:, j]) ** 2, -1))
    v_ne = np.zeros(B)
    for i in range(N):
        for m in range(M):
            v_ne -= charges[m] / np.sqrt(np.sum((r[:, i] - nuclei[m]) ** 2, -1))
    v_nn = 0.0
    for m in range(M):
        for n in range(m + 1, M):
            v_nn += charges[m] * charges[n] / np.sqrt(np.sum((nuclei[m] - nuclei[n]) ** 2))
    return v_ee, v_ne, np.full(B, v_nn)


def local_energy(net: Net, params: np.ndarray, nuclei: np.ndarray, charges: np.ndarray,
                 r: np.ndarray):
    """(E_L, log|psi|, sign) per walker, exact Laplacian (Eqs. 2-3)."""
    lpsi, sign, grad, lap = log_psi_derivatives(net, params, nuclei, r)
    v_ee, v_ne, v_nn = potential_energy(nuclei, charges, r)
    kinetic = -0.5 * (np.sum(grad * grad, -1) + lap)
    return kinetic + v_ee + v_ne + v_nn, lpsi, sign


def fd_log_psi_derivatives(net: Net, params: np.ndarray, nuclei: np.ndarray, r: np.ndarray,
                           h: float = 1e-4):
    """Central differences of log|psi|: gradient [B, 3N] and Laplacian [B]."""
    r = np.asarray(r, dtype=np.float64)
    B, N, _ = r.shape
    f0, _ = log_psi(net, params, nuclei, r)
    grad = np.zeros((B, 3 * N))
    lap = np.zeros(B)
    for e in range(N):
        for c in range(3):
            rp = r.copy()
            rp[:, e, c] += h
            rm = r.copy()
            rm[:, e, c] -= h
            fp, _ = log_psi(net, params, nuclei, rp)
            fm, _ = log_psi(net, params, nuclei, rm)
            grad[:, 3 * e + c] = (fp - fm) / (2 * h)
            lap += (fp - 2 * f0 + fm) / (h * h)
    return f0, grad, lap
