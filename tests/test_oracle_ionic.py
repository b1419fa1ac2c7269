"""Pins of Algorithm 1 and the spin split."""
import os

import numpy as np
import pytest

from oracle import ionic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            out[k] = v
    return out


def test_worked_example_lih_cation():
    g = _read_golden("algorithm1_lih_cation.txt")
    counts = ionic.ionic_electron_counts([int(v) for v in g["atomic_numbers"]],
                                         [float(v) for v in g["partial_charges"]],
                                         int(g["total_charge"][0]))
    assert counts == [int(v) for v in g["expected_counts"]]


def test_neutral_is_atomic_numbers():
    assert ionic.ionic_electron_counts([7, 7], [0.1, -0.1], 0) == [7, 7]


@pytest.mark.parametrize("seed", range(20))
def test_invariants_random(seed):
    rs = np.random.default_rng(seed)
    m = int(rs.integers(1, 6))
    z = [int(v) for v in rs.integers(1, 15, m)]
    t = int(rs.integers(-4, 5))
    t = min(t, sum(z))
    q = list(rs.normal(size=m))
    counts = ionic.ionic_electron_counts(z, q, t)
    assert sum(counts) == sum(z) - t
    assert all(c >= 0 for c in counts)
    assert all(isinstance(c, int) for c in counts)
    # each atom changes by at most |t| and only in the direction of the charge
    for c, zz in zip(counts, z):
        assert (c - zz) * (-t) >= 0
        assert abs(c - zz) <= abs(t)


def test_anion_goes_to_most_negative_then_spreads():
    # charges -0.3, -0.2: first electron to atom 0 (its charge becomes 0.7), second to atom 1
    assert ionic.ionic_electron_counts([1, 1], [-0.3, -0.2], -2) == [2, 2]
    # cation: highest partial charge loses first, its charge drops by 1, next goes elsewhere
    assert ionic.ionic_electron_counts([3, 1], [0.6, 0.4], 2) == [2, 0]


def test_ties_lowest_index_and_fallback():
    assert ionic.ionic_electron_counts([3, 1], None, -1) == [4, 1]
    assert ionic.ionic_electron_counts([3, 1], None, 1) == [2, 1]
    assert ionic.ionic_electron_counts([1], None, 1) == [0]


def test_empty_atom_not_eligible_and_error():
    # H loses its electron first (largest charge), then Li must give the next one
    assert ionic.ionic_electron_counts([3, 1], [0.1, 0.9], 2) == [2, 0]
    with pytest.raises(ValueError):
        ionic.ionic_electron_counts([1], None, 2)


def test_spin_split_and_order():
    up, dn = ionic.spin_split([2, 1], 2, 1)          # LiH+
    assert (up, dn) == ([1, 1], [1, 0])
    up, dn = ionic.spin_split([4, 1], 3, 2)          # LiH-
    assert (up, dn) == ([2, 1], [2, 0])
    up, dn = ionic.spin_split([1, 1], 2, 0)          # triplet H2: no flip needed
    assert (up, dn) == ([1, 1], [0, 0])
    up, dn = ionic.spin_split([1, 1], 1, 1)          # H2 singlet: tie in (up - down), atom 0 flips
    assert (up, dn) == ([0, 1], [1, 0])
    assert list(ionic.electron_atoms([1, 1], 1, 1)) == [1, 0]
    up, dn = ionic.spin_split([7, 7], 7, 7)          # N2: atom 0 flips first
    assert (up, dn) == ([3, 4], [4, 3])
    assert list(ionic.electron_atoms([4, 1], 3, 2)) == [0, 0, 1, 0, 0]
