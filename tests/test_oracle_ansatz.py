"""Pins of the oracle wavefunction and local energy: closed forms, brute force, library LU, FD."""
import itertools
import os

import numpy as np
import pytest

import workloads as W
from oracle import ansatz, mcmc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _net(sysm, L=2, h1=16, h2=8, K=2, env="aniso"):
    return ansatz.Net(sysm.nuclei.shape[0], sysm.n_up, sysm.n_down, L, h1, h2, K, env)


def _walkers(sysm, B, seed=0, std=1.0):
    r, _ = mcmc.init_walkers(sysm.nuclei, sysm.charges, sysm.n_up, sysm.n_down,
                             sysm.partial_charges, B, seed, std)
    return r


def _perturbed(net, seed=0, scale=0.1):
    p = ansatz.init_params(net, seed)
    return p + scale * np.random.default_rng(seed).standard_normal(p.shape)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_lu_against_library(n):
    a = np.random.default_rng(n).standard_normal((40, n, n))
    s, ld = ansatz.slogdet(a)
    s_ref, ld_ref = np.linalg.slogdet(a)
    np.testing.assert_array_equal(s, s_ref)
    np.testing.assert_allclose(ld, ld_ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ansatz.inverse(a), np.linalg.inv(a), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_det_leibniz_brute_force(n):
    a = np.random.default_rng(10 + n).standard_normal((20, n, n))
    det = np.zeros(20)
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        det += (-1) ** inv * np.prod([a[:, i, perm[i]] for i in range(n)], axis=0)
    s, ld = ansatz.slogdet(a)
    np.testing.assert_allclose(s * np.exp(ld), det, rtol=1e-12, atol=1e-14)


def _set(net, blob, **kw):
    p = ansatz.unpack(net, blob)
    for k, v in kw.items():
        p[k][...] = v
    return blob


@pytest.mark.parametrize("env", ["iso", "aniso"])
def test_hydrogen_atom_zero_variance(env):
    """w = 0, g = 1, pi = 1, sigma = 1: psi = exp(-r) and E_L = -1/2 everywhere."""
    s = W.hydrogen_atom()
    net = ansatz.Net(1, 1, 0, 2, 16, 8, 1, env)
    blob = _set(net, ansatz.init_params(net, 3), w_up=0.0, g_up=1.0)
    r = _walkers(s, 64, seed=2)
    e, lp, sign = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
    np.testing.assert_allclose(e, -0.5, atol=1e-12)
    np.testing.assert_allclose(lp, -np.linalg.norm(r[:, 0], axis=-1), atol=1e-13)
    assert np.all(sign == 1)


@pytest.mark.parametrize("zeta", [0.7, 1.3])
def test_hydrogenic_closed_form(zeta):
    """psi = exp(-zeta r): E_L = -zeta^2/2 + (zeta - 1)/r; also via sigma = zeta * I (aniso)."""
    s = W.hydrogen_atom()
    r = _walkers(s, 64, seed=5)
    rad = np.linalg.norm(r[:, 0], axis=-1)
    for env, sig in (("iso", zeta), ("aniso", zeta * np.eye(3))):
        net = ansatz.Net(1, 1, 0, 1, 8, 4, 1, env)
        blob = _set(net, ansatz.init_params(net, 4), w_up=0.0, g_up=2.0, sigma_up=sig)
        e, lp, _ = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
        np.testing.assert_allclose(e, -zeta ** 2 / 2 + (zeta - 1) / rad, rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(lp, np.log(2.0) - zeta * rad, atol=1e-12)


def test_two_electron_atom_closed_form():
    """He-like product exp(-zeta r1) exp(-zeta r2), 1 up + 1 down:
    E_L = -zeta^2 + (zeta - Z)(1/r1 + 1/r2) + 1/r12."""
    Z, zeta = 2.0, 1.6875
    s = W.System("He", np.zeros((1, 3)), np.array([Z]), 1, 1)
    net = ansatz.Net(1, 1, 1, 2, 8, 4, 1, "iso")
    blob = _set(net, ansatz.init_params(net, 1), w_up=0.0, g_up=1.0, w_down=0.0, g_down=1.0,
                sigma_up=zeta, sigma_down=zeta)
    r = _walkers(s, 64, seed=3)
    r1, r2 = np.linalg.norm(r[:, 0], axis=-1), np.linalg.norm(r[:, 1], axis=-1)
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=-1)
    e, _, _ = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
    np.testing.assert_allclose(e, -zeta ** 2 + (zeta - Z) * (1 / r1 + 1 / r2) + 1 / r12, rtol=1e-11)


def test_nuclear_repulsion_golden():
    systems = {"H2": W.h2(), "N2": W.n2(), "LiH": W.lih(0), "CO": W.co()}
    with open(os.path.join(GOLDEN, "nuclear_repulsion.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, _, _, _, num, den = line.split()
            s = systems[name]
            _, _, v_nn = ansatz.potential_energy(s.nuclei, s.charges, np.zeros((1, 1, 3)) + 5.0)
            assert abs(v_nn[0] - float(num) / float(den)) < 1e-13


@pytest.mark.parametrize("make", [W.n2, lambda: W.lih(-1), lambda: W.lih(1)])
def test_antisymmetry_same_spin(make):
    s = make()
    net = _net(s, L=3, h1=16, h2=8, K=3)
    blob = _perturbed(net)
    r = _walkers(s, 16)
    lp, sg = ansatz.log_psi(net, blob, s.nuclei, r)
    pairs = [(0, 1)] + ([(s.n_up, s.n_up + 1)] if s.n_down >= 2 else [])
    for a, b in pairs:
        rs = r.copy()
        rs[:, [a, b]] = rs[:, [b, a]]
        lp2, sg2 = ansatz.log_psi(net, blob, s.nuclei, rs)
        np.testing.assert_allclose(lp2, lp, atol=1e-12, rtol=1e-12)
        np.testing.assert_array_equal(sg2, -sg)


@pytest.mark.parametrize("make,env", [(W.h2, "iso"), (lambda: W.lih(1), "aniso"),
                                      (lambda: W.lih(-1), "aniso"), (W.hydrogen_atom, "aniso")])
def test_forward_laplacian_against_finite_differences(make, env):
    """Richardson-extrapolated central differences (h, h/2) against the exact jets."""
    s = make()
    net = _net(s, L=3, h1=12, h2=6, K=2, env=env)
    blob = _perturbed(net, seed=7)
    r = _walkers(s, 6, seed=8)
    lp, _, grad, lap = ansatz.log_psi_derivatives(net, blob, s.nuclei, r)
    _, g1, l1 = ansatz.fd_log_psi_derivatives(net, blob, s.nuclei, r, 4e-4)
    f0, g2, l2 = ansatz.fd_log_psi_derivatives(net, blob, s.nuclei, r, 2e-4)
    g_ex = (4 * g2 - g1) / 3
    l_ex = (4 * l2 - l1) / 3
    np.testing.assert_allclose(lp, f0, atol=1e-13)
    np.testing.assert_allclose(grad, g_ex, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(lap, l_ex, rtol=1e-5, atol=1e-4)


def test_three_electron_leibniz_brute_force():
    """2 up + 1 down: psi = sum_k det2(A_up^k) A_down^k by explicit products, no LU."""
    s = W.lih(1)
    net = _net(s, L=2, h1=8, h2=4, K=3, env="aniso")
    blob = _perturbed(net, seed=3)
    r = _walkers(s, 10)
    a_up, a_dn = ansatz.orbital_matrices(net, blob, s.nuclei, r)
    det_up = a_up[..., 0, 0] * a_up[..., 1, 1] - a_up[..., 0, 1] * a_up[..., 1, 0]
    psi = np.sum(det_up * a_dn[..., 0, 0], axis=-1)
    lp, sg = ansatz.log_psi(net, blob, s.nuclei, r)
    np.testing.assert_allclose(lp, np.log(np.abs(psi)), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(sg, np.sign(psi))


def test_two_electron_brute_force_energy():
    """1 up + 1 down: psi = sum_k phi_up^k(r1) phi_down^k(r2); its Laplacian by FD of log psi."""
    s = W.h2()
    net = _net(s, L=2, h1=8, h2=4, K=3, env="iso")
    blob = _perturbed(net, seed=9)
    r = _walkers(s, 8)

    def brute(rr):
        a_up, a_dn = ansatz.orbital_matrices(net, blob, s.nuclei, rr)
        return np.log(np.abs(np.sum(a_up[..., 0, 0] * a_dn[..., 0, 0], axis=-1)))

    h = 2e-4
    f0 = brute(r)
    lap = np.zeros(r.shape[0])
    for e in range(2):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[:, e, c] += h
            rm[:, e, c] -= h
            lap += (brute(rp) - 2 * f0 + brute(rm)) / h ** 2
    lp, _, grad, lap_jet = ansatz.log_psi_derivatives(net, blob, s.nuclei, r)
    np.testing.assert_allclose(lp, f0, atol=1e-12)
    np.testing.assert_allclose(lap_jet, lap, rtol=1e-4, atol=1e-4)


def test_init_params_statistics():
    s = W.n2()
    net = ansatz.Net(2, 7, 7, 4, 256, 32, 16, "aniso")
    blob = ansatz.init_params(net, 1)
    p = ansatz.unpack(net, blob)
    for name, shape, fan_in, kind in ansatz.param_layout(net):
        if kind == "normal" and p[name].size > 2000:
            x = p[name] * np.sqrt(fan_in)
            assert abs(x.mean()) < 0.05 and abs(x.std() - 1) < 0.05, name
    assert np.all(p["pi_up"] == 1.0)
    np.testing.assert_array_equal(p["sigma_down"][3, 1], np.eye(3))
    assert ansatz.param_count(net) == blob.shape[0]


@pytest.mark.parametrize("make,env", [(W.n2, "aniso"), (lambda: W.lih(1), "iso"), (lambda: W.atom(6), "aniso")])
def test_translation_invariance(make, env):
    """The method sees positions only as differences: the one-electron features use r_i - R_m,
    the pair features r_i - r_j, the envelopes of Eq. 4 act on r_j - R_m, and the Coulomb terms
    on distances.  Moving every nucleus and electron by the same vector therefore leaves
    log|psi|, its sign and E_L unchanged (up to the rounding of the shifted coordinates)."""
    s = make()
    net = _net(s, L=3, h1=16, h2=8, K=2, env=env)
    blob = _perturbed(net, seed=11)
    r = _walkers(s, 8, seed=12)
    shift = np.array([0.75, -1.25, 2.5])
    e0, lp0, sg0 = ansatz.local_energy(net, blob, s.nuclei, s.charges, r)
    e1, lp1, sg1 = ansatz.local_energy(net, blob, s.nuclei + shift, s.charges, r + shift)
    np.testing.assert_array_equal(sg1, sg0)
    np.testing.assert_allclose(lp1, lp0, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(e1, e0, rtol=1e-8, atol=1e-8)
