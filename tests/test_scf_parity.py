"""fn_mulliken_charges (host code of the library: Obara-Saika integrals, the published STO-6G
table) against the oracle (McMurchie-Davidson integrals, STO-6G fitted from scratch).  The
entry point makes no CUDA call, so these tests run without a GPU.  The two STO-6G tables agree
to about 1e-5, which bounds the agreement of the energies (1e-6 Ha) and charges (1e-6)."""
import os

import numpy as np
import pytest

from oracle import ionic, scf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def P():
    from paper_2401_10287_gb300 import build
    build.build()
    import paper_2401_10287_gb300 as pkg
    return pkg


def _rot(nuc, seed):
    rs = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rs.standard_normal((3, 3)))
    return np.asarray(nuc, float) @ q.T + rs.standard_normal(3)


CASES = {
    "H": ([[0, 0, 0]], [1], 1, 0),
    "H2": ([[0, 0, 0], [0, 0, 1.4]], [1, 1], 1, 1),
    "HeH+": ([[0, 0, 0], [0, 0, 1.46]], [2, 1], 1, 1),
    "LiH": ([[0, 0, 0], [0, 0, 3.015]], [3, 1], 2, 2),
    "LiH+": ([[0, 0, 0], [0, 0, 3.015]], [3, 1], 2, 1),
    "LiH-": ([[0, 0, 0], [0, 0, 3.015]], [3, 1], 3, 2),
    "BeH": ([[0, 0, 0], [0, 0, 2.54]], [4, 1], 3, 2),
    "OH-": ([[0, 0, 0], [0.3, 0.5, 1.7]], [8, 1], 5, 5),
    "N2": ([[0, 0, -1.034], [0, 0, 1.034]], [7, 7], 7, 7),
    "CO+": (_rot([[0, 0, 0], [0, 0, 2.132]], 3), [6, 8], 7, 6),
    "H2O": ([[0, 0, 0], [1.43, 1.11, 0], [-1.43, 1.11, 0]], [8, 1, 1], 5, 5),
    "F2": ([[0, 0, 0], [0, 0, 2.68]], [9, 9], 9, 9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mulliken_charges_match_oracle(P, name):
    nuc, z, nu, nd = CASES[name]
    q, e = P.mulliken_charges(np.asarray(nuc, float), z, nu, nd)
    q_ref, e_ref = scf.mulliken_charges(np.asarray(nuc, float), z, nu, nd)
    np.testing.assert_allclose(q, q_ref, atol=1e-6)
    assert e == pytest.approx(e_ref, abs=1e-6)
    assert q.sum() == pytest.approx(sum(z) - nu - nd, abs=1e-10)


def test_printed_lih_cation_example_and_algorithm1(P):
    vals = {}
    with open(os.path.join(GOLDEN, "lih_cation_mulliken.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                vals[k] = [float(x) for x in v]
    R = vals["internuclear_distance_bohr"][0]
    q, _ = P.mulliken_charges(np.array([[0, 0, 0], [0, 0, R]]), [3, 1], 2, 1)
    np.testing.assert_allclose(q, vals["charges"], atol=vals["tolerance"][0])
    assert ionic.ionic_electron_counts([3, 1], list(q), 1) == [2, 1]


def test_spin_labels_and_rotation_do_not_matter(P):
    nuc = np.array([[0, 0, 0], [0, 0, 3.015]])
    q1, e1 = P.mulliken_charges(nuc, [3, 1], 2, 1)
    q2, e2 = P.mulliken_charges(nuc, [3, 1], 1, 2)
    q3, e3 = P.mulliken_charges(_rot(nuc, 7), [3, 1], 2, 1)
    np.testing.assert_allclose(q2, q1, atol=1e-12)
    np.testing.assert_allclose(q3, q1, atol=1e-8)
    assert e3 == pytest.approx(e1, abs=1e-9)


def test_arguments_outside_the_basis_are_refused(P):
    with pytest.raises(P.FnError) as err:
        P.mulliken_charges(np.zeros((1, 3)), [11], 6, 5)                 # Na: no STO-6G 3sp shell here
    assert err.value.code == 1
    with pytest.raises(P.FnError) as err:                                 # 5 carbons: 25 functions
        P.mulliken_charges(np.arange(15, dtype=float).reshape(5, 3), [6] * 5, 15, 15)
    assert err.value.code == 7
    with pytest.raises(P.FnError) as err:
        P.mulliken_charges(np.zeros((1, 3)), [1], 0, 0)
    assert err.value.code == 1
    with pytest.raises(P.FnError) as err:                                 # He-: two up electrons, one function
        P.mulliken_charges(np.zeros((1, 3)), [2], 2, 1)
    assert err.value.code == 1
    with pytest.raises(P.FnError) as err:                                 # coincident nuclei
        P.mulliken_charges(np.zeros((2, 3)), [1, 1], 1, 1)
    assert err.value.code == 1


def test_algorithm1_on_library_charges_of_ions(P):
    """CO+: C carries the most positive charge, so Algorithm 1 removes the electron from C;
    OH-: O carries the most negative one and receives the extra electron."""
    q, _ = P.mulliken_charges(np.array([[0, 0, 0], [0, 0, 2.132]]), [6, 8], 7, 6)
    assert q[0] > q[1] > 0
    assert ionic.ionic_electron_counts([6, 8], list(q), 1) == [5, 8]
    q, _ = P.mulliken_charges(np.array([[0, 0, 0], [0.3, 0.5, 1.7]]), [8, 1], 5, 5)
    assert q[0] < q[1] < 0
    assert ionic.ionic_electron_counts([8, 1], list(q), -1) == [9, 1]
