"""Pins of the Eq. 5 pretraining oracle: the basis values (normalisation by radial quadrature,
Laplacians against finite differences), the occupied HF orbitals (Roothaan-Hall equations,
orthonormality, the energy recomputed from them), the determinant convention (antisymmetry)
and the variational identity <E_L>_{|psi_HF|^2} = E_HF."""
import numpy as np
import pytest

import workloads as W
from oracle import ansatz, pretrain


@pytest.fixture(scope="module")
def lih():
    s = W.lih(0)
    return s, pretrain.hf_state(s.nuclei, s.charges, s.n_up, s.n_down)


def test_basis_functions_are_normalised_by_radial_quadrature(lih):
    """s: 4 pi int chi(A + r e)^2 r^2 dr; p_a along its own axis: (4 pi / 3) int chi^2 r^2 dr."""
    _, st = lih
    x, w = np.polynomial.legendre.leggauss(2000)
    t = 0.5 * (x + 1)
    r = t / (1 - t)
    wr = 0.5 * w / (1 - t) ** 2
    for mu, f in enumerate(st["basis"]):
        axis = int(np.argmax(f.lmn)) if sum(f.lmn) else 2
        e = np.zeros(3)
        e[axis] = 1.0
        chi = pretrain.basis_values(st["basis"], f.centre + r[:, None] * e)[:, mu]
        fac = 4 * np.pi / (3 if sum(f.lmn) else 1)
        assert fac * np.sum(wr * chi * chi * r * r) == pytest.approx(1.0, abs=1e-10), mu


def test_basis_laplacians_match_finite_differences(lih):
    _, st = lih
    pts = np.random.default_rng(0).normal(0.0, 1.2, (20, 3)) + np.array([0, 0, 1.0])
    h = 1e-4
    fd = np.zeros((20, len(st["basis"])))
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd += (pretrain.basis_values(st["basis"], pts + e) - 2 * pretrain.basis_values(st["basis"], pts)
               + pretrain.basis_values(st["basis"], pts - e)) / (h * h)
    np.testing.assert_allclose(pretrain.basis_laplacians(st["basis"], pts), fd, rtol=1e-5, atol=1e-5)


def test_occupied_orbitals_solve_roothaan_hall_and_give_the_energy(lih):
    _, st = lih
    S = st["S"]
    P = {}
    for spin in ("up", "down"):
        C, eps, F = st[f"C_{spin}"], st[f"eps_{spin}"], st[f"F_{spin}"]
        np.testing.assert_allclose(F @ C, S @ C * eps, atol=1e-7)
        np.testing.assert_allclose(C.T @ S @ C, np.eye(C.shape[1]), atol=1e-10)
        P[spin] = C @ C.T
    e = 0.5 * (np.sum((st["H"] + st["F_up"]) * P["up"]) + np.sum((st["H"] + st["F_down"]) * P["down"])) + st["e_nn"]
    assert e == pytest.approx(st["energy"], abs=1e-7)   # the SCF stops at a commutator of 1e-8
    for spin in ("up", "down"):          # sign convention: largest coefficient positive
        C = st[f"C_{spin}"]
        assert np.all(C[np.argmax(np.abs(C), 0), np.arange(C.shape[1])] > 0)


def test_hf_determinant_is_antisymmetric(lih):
    s, st = lih
    r = np.random.default_rng(1).normal(0.0, 1.0, (5, 4, 3))
    up, down = pretrain.hf_orbital_matrices(st, r)
    r2 = r.copy()
    r2[:, [0, 1]] = r2[:, [1, 0]]          # swap the two up electrons
    up2, down2 = pretrain.hf_orbital_matrices(st, r2)
    np.testing.assert_allclose(np.linalg.det(up2), -np.linalg.det(up), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(down2, down, atol=0)


def test_variational_identity_h2():
    """<E_L> of the HF determinant over |psi_HF|^2 is the UHF energy (within 5 standard errors of
    the mean over walkers)."""
    s = W.h2()
    st = pretrain.hf_state(s.nuclei, s.charges, 1, 1)
    r = pretrain.sample_hf(st, s.nuclei, s.charges, 1, 1, 3000, 150, 0.3, 3)
    e = pretrain.hf_local_energy(st, s.nuclei, s.charges, r)
    assert abs(e.mean() - st["energy"]) < 5 * e.std() / np.sqrt(e.size)


def test_loss_is_the_mean_over_walkers_of_the_squared_differences(lih):
    s, st = lih
    r = np.random.default_rng(2).normal(0.0, 1.0, (3, 4, 3)) + np.array([0, 0, 1.0])
    hf = pretrain.hf_orbital_matrices(st, r)
    K = 2
    same = [np.repeat(h[:, None], K, axis=1) for h in hf]
    assert pretrain.pretrain_loss_from(same, hf) == 0.0
    bumped = [x.copy() for x in same]
    bumped[1][2, 1, 0, 1] += 0.3
    assert pretrain.pretrain_loss_from(bumped, hf) == pytest.approx(0.09 / 3, abs=1e-15)
    net = ansatz.Net(2, 2, 2, 2, 8, 4, K, "aniso")
    p = ansatz.init_params(net, 0)
    assert pretrain.pretrain_loss(net, p, s.nuclei, r, st) == pytest.approx(
        pretrain.pretrain_loss_from(ansatz.orbital_matrices(net, p, s.nuclei, r), hf), abs=1e-12)


def test_degenerate_occupied_level_is_refused():
    """N2: the occupied pi levels are degenerate, so their orbitals are not unique."""
    s = W.n2()
    with pytest.raises(ValueError):
        pretrain.hf_state(s.nuclei, s.charges, s.n_up, s.n_down)
