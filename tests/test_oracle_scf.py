"""Pins of the oracle's STO-6G Hartree-Fock and Mulliken charges (the partial charges that
Algorithm 1 takes).  Integrals over s functions are checked against textbook closed forms
typed here; integrals with p functions against centre derivatives of those closed forms
(a normalised p_x primitive at A is (1/sqrt(a)) d/dA_x of the normalised s primitive);
the energy of the hydrogen atom against radial quadrature; the charges against the
example the paper prints."""
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import ionic, scf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prim(centre, a, lmn=(0, 0, 0)):
    return scf.Contracted(np.asarray(centre, np.float64), lmn, np.array([a]), np.array([1.0]), 0)


# closed forms for normalised s primitives
def _ns(a):
    return (2 * a / np.pi) ** 0.75


def _f0(t):
    return 1.0 if t < 1e-14 else 0.5 * math.sqrt(math.pi / t) * math.erf(math.sqrt(t))


def s_overlap(A, a, B, b):
    p, q = a + b, a * b / (a + b)
    return _ns(a) * _ns(b) * (np.pi / p) ** 1.5 * math.exp(-q * np.sum((A - B) ** 2))


def s_kinetic(A, a, B, b):
    q = a * b / (a + b)
    r2 = np.sum((A - B) ** 2)
    return q * (3 - 2 * q * r2) * s_overlap(A, a, B, b)


def s_nuclear(A, a, B, b, C):
    p, q = a + b, a * b / (a + b)
    P = (a * A + b * B) / p
    return _ns(a) * _ns(b) * 2 * np.pi / p * math.exp(-q * np.sum((A - B) ** 2)) * _f0(p * np.sum((P - C) ** 2))


def s_eri(A, a, B, b, C, c, D, d):
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    k = math.exp(-a * b / p * np.sum((A - B) ** 2) - c * d / q * np.sum((C - D) ** 2))
    al = p * q / (p + q)
    return _ns(a) * _ns(b) * _ns(c) * _ns(d) * 2 * np.pi ** 2.5 / (p * q * math.sqrt(p + q)) * k * \
        _f0(al * np.sum((P - Q) ** 2))


A, B, C, D = (np.array(x) for x in ([0.1, -0.2, 0.3], [0.7, 0.4, -0.5], [-0.6, 0.2, 0.9], [0.3, 0.8, 0.1]))
a, b, c, d = 1.3, 0.45, 2.1, 0.8


def test_s_integrals_equal_closed_forms():
    fa, fb, fc, fd = _prim(A, a), _prim(B, b), _prim(C, c), _prim(D, d)
    assert scf.overlap(fa, fb) == pytest.approx(s_overlap(A, a, B, b), rel=1e-13)
    assert scf.kinetic(fa, fb) == pytest.approx(s_kinetic(A, a, B, b), rel=1e-12)
    assert scf.nuclear(fa, fb, C) == pytest.approx(s_nuclear(A, a, B, b, C), rel=1e-12)
    assert scf.eri(fa, fb, fc, fd) == pytest.approx(s_eri(A, a, B, b, C, c, D, d), rel=1e-12)
    assert scf.boys(0, 0.0) == 1.0 and scf.boys(2, 0.0) == pytest.approx(0.2)


def _d(fun, X, axis, h):
    e = np.zeros(3)
    e[axis] = h
    return (fun(X + e) - fun(X - e)) / (2 * h)


AX = {"x": 0, "y": 1, "z": 2}
LMN = {"x": (1, 0, 0), "y": (0, 1, 0), "z": (0, 0, 1)}


@pytest.mark.parametrize("ax", ["x", "y", "z"])
def test_one_p_function_is_a_centre_derivative(ax):
    i, h = AX[ax], 1e-4
    pa = _prim(A, a, LMN[ax])
    fb, fc, fd = _prim(B, b), _prim(C, c), _prim(D, d)
    ref_s = _d(lambda X: s_overlap(X, a, B, b), A, i, h) / math.sqrt(a)
    ref_t = _d(lambda X: s_kinetic(X, a, B, b), A, i, h) / math.sqrt(a)
    ref_v = _d(lambda X: s_nuclear(X, a, B, b, C), A, i, h) / math.sqrt(a)
    ref_g = _d(lambda X: s_eri(X, a, B, b, C, c, D, d), A, i, h) / math.sqrt(a)
    assert scf.overlap(pa, fb) == pytest.approx(ref_s, rel=1e-7, abs=1e-10)
    assert scf.kinetic(pa, fb) == pytest.approx(ref_t, rel=1e-7, abs=1e-10)
    assert scf.nuclear(pa, fb, C) == pytest.approx(ref_v, rel=1e-7, abs=1e-10)
    assert scf.eri(pa, fb, fc, fd) == pytest.approx(ref_g, rel=1e-7, abs=1e-10)
    # the p function in the other slots of the two-electron integral
    assert scf.eri(fb, pa, fc, fd) == pytest.approx(ref_g, rel=1e-7, abs=1e-10)
    assert scf.eri(fc, fd, pa, fb) == pytest.approx(ref_g, rel=1e-7, abs=1e-10)


@pytest.mark.parametrize("ax1,ax2", [("x", "x"), ("x", "z"), ("z", "y"), ("z", "z")])
def test_two_p_functions_are_mixed_centre_derivatives(ax1, ax2):
    i, j, h = AX[ax1], AX[ax2], 1e-3
    pa, pb = _prim(A, a, LMN[ax1]), _prim(B, b, LMN[ax2])
    pc = _prim(C, c, LMN[ax2])
    fb, fc, fd = _prim(B, b), _prim(C, c), _prim(D, d)

    def mixed(fun):   # d^2 / dA_i de_j of fun(A, e), e the shift of the second centre
        tot = 0.0
        for sa, sy in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            ea, ey = np.zeros(3), np.zeros(3)
            ea[i], ey[j] = sa * h, sy * h
            tot += sa * sy * fun(A + ea, ey)
        return tot / (4 * h * h)

    ref_s = mixed(lambda X, e: s_overlap(X, a, B + e, b)) / math.sqrt(a * b)
    ref_t = mixed(lambda X, e: s_kinetic(X, a, B + e, b)) / math.sqrt(a * b)
    ref_v = mixed(lambda X, e: s_nuclear(X, a, B + e, b, C)) / math.sqrt(a * b)
    ref_g = mixed(lambda X, e: s_eri(X, a, B, b, C + e, c, D, d)) / math.sqrt(a * c)
    assert scf.overlap(pa, pb) == pytest.approx(ref_s, rel=1e-5, abs=1e-8)
    assert scf.kinetic(pa, pb) == pytest.approx(ref_t, rel=1e-5, abs=1e-8)
    assert scf.nuclear(pa, pb, C) == pytest.approx(ref_v, rel=1e-5, abs=1e-8)
    assert scf.eri(pa, fb, pc, fd) == pytest.approx(ref_g, rel=1e-5, abs=1e-8)


def test_eri_symmetry_and_normalisation():
    nuc = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.2]])
    basis = scf.sto6g_basis([3, 1], nuc)
    S, H, G, _ = scf.integrals(basis, nuc, [3, 1])
    np.testing.assert_allclose(np.diag(S), 1.0, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(S) > 0)
    f = basis
    for (i, j, k, l) in ((1, 2, 3, 5), (4, 0, 2, 2), (3, 3, 4, 1)):
        x = scf.eri(f[i], f[j], f[k], f[l])
        for y in (scf.eri(f[j], f[i], f[k], f[l]), scf.eri(f[k], f[l], f[i], f[j]), scf.eri(f[l], f[k], f[j], f[i])):
            assert y == pytest.approx(x, rel=1e-12, abs=1e-15)
        assert G[i, j, k, l] == pytest.approx(x, rel=1e-12, abs=1e-15)
    # Schwarz inequality
    for i in range(len(f)):
        for k in range(len(f)):
            assert abs(G[i, i, k, k]) <= math.sqrt(G[i, i, i, i] * G[k, k, k, k]) + 1e-12


def test_hydrogen_atom_energy_by_radial_quadrature():
    """One electron: E = <phi| -1/2 nabla^2 - 1/r |phi> of the contracted 1s (zeta 1.24),
    integrated on a radial grid from the expansion alone."""
    q, e = scf.mulliken_charges(np.zeros((1, 3)), [1], 1, 0)
    exps, (coef,) = scf.sto6g_expansion("1s")
    a = exps * 1.24 ** 2
    x, w = np.polynomial.legendre.leggauss(4000)
    t = 0.5 * (x + 1)
    r = t / (1 - t)
    wr = 0.5 * w / (1 - t) ** 2
    nrm = (2 * a / np.pi) ** 0.75
    phi = np.sum(coef[:, None] * nrm[:, None] * np.exp(-a[:, None] * r * r), 0)
    dphi = np.sum(coef[:, None] * nrm[:, None] * (-2 * a[:, None] * r) * np.exp(-a[:, None] * r * r), 0)
    norm = np.sum(wr * 4 * np.pi * r * r * phi * phi)
    e_ref = (np.sum(wr * 4 * np.pi * r * r * 0.5 * dphi * dphi) - np.sum(wr * 4 * np.pi * r * phi * phi)) / norm
    assert e == pytest.approx(e_ref, abs=1e-10)
    assert abs(q[0]) < 1e-12


def test_charges_are_rotation_invariant_and_sum_to_the_ionic_charge():
    R = 1.8
    q1, e1 = scf.mulliken_charges(np.array([[0, 0, 0], [0, 0, R]]), [3, 1], 2, 1)
    u = np.array([1.0, -2.0, 0.5])
    u /= np.linalg.norm(u)
    q2, e2 = scf.mulliken_charges(np.array([[0.2, 0.1, -0.3], [0.2, 0.1, -0.3] + R * u]), [3, 1], 2, 1)
    assert e2 == pytest.approx(e1, abs=1e-9)
    np.testing.assert_allclose(q2, q1, atol=1e-8)
    assert q1.sum() == pytest.approx(1.0, abs=1e-10)


def _golden():
    out = {}
    with open(os.path.join(GOLDEN, "lih_cation_mulliken.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out[k] = [float(x) for x in v]
    return out


def test_lih_cation_charges_match_the_printed_example():
    g = _golden()
    R = g["internuclear_distance_bohr"][0]
    q, _ = scf.mulliken_charges(np.array([[0, 0, 0], [0, 0, R]]), [3, 1], 2, 1)
    np.testing.assert_allclose(q, g["charges"], atol=g["tolerance"][0])
    # and Algorithm 1 on them removes the cation's electron from Li
    assert ionic.ionic_electron_counts([3, 1], list(q), 1) == [2, 1]


def test_n2_ground_state_has_degenerate_pi_levels():
    """The D_inf_h ground state occupies both pi_u orbitals at one energy.  An excited
    self-consistent solution that DIIS from the core guess settles on (-107.818 Ha) breaks this."""
    import workloads as W
    s = W.n2()
    basis = scf.sto6g_basis(s.charges, s.nuclei)
    S, H, G, e_nn = scf.integrals(basis, s.nuclei, s.charges)
    e, Pa, Pb = scf.uhf(S, H, G, 7, 7, e_nn)
    sv, U = np.linalg.eigh(S)
    X = U @ np.diag(sv ** -0.5) @ U.T
    F = H + np.einsum("pqrs,rs->pq", G, Pa + Pb) - np.einsum("prqs,rs->pq", G, Pa)
    eps = np.linalg.eigvalsh(X.T @ F @ X)
    occ = eps[:7]
    assert np.min(np.abs(np.subtract.outer(occ, occ)) + 10 * np.eye(7)) < 1e-7     # a degenerate pair
    assert eps[7] - eps[6] > 0.5                                                    # a clear gap
    assert e == pytest.approx(-108.5408098, abs=1e-6)


@pytest.mark.parametrize("name", ["N2", "CO+"])
def test_uhf_energy_is_the_lowest_over_random_starts(name):
    """Damped iterations from randomised starting Fock matrices never reach a lower energy."""
    nuc = {"N2": [[0, 0, -1.034], [0, 0, 1.034]], "CO+": [[0, 0, 0], [0, 0, 2.132]]}[name]
    z, na, nb = {"N2": ([7, 7], 7, 7), "CO+": ([6, 8], 7, 6)}[name]
    nuc = np.asarray(nuc, float)
    basis = scf.sto6g_basis(z, nuc)
    S, H, G, e_nn = scf.integrals(basis, nuc, z)
    e_best, _, _ = scf.uhf(S, H, G, na, nb, e_nn)
    rs = np.random.default_rng(5)
    for _ in range(4):
        A = rs.standard_normal(H.shape)
        F0 = H + 0.3 * (A + A.T)
        e, _, _ = scf._uhf_from(F0, S, H, G, na, nb, e_nn, 1e-10, 2000, 2000)
        assert e >= e_best - 1e-7
