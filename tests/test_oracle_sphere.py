"""Pins of the oracle's plane-wave sphere (Sec. 3.2.2 item (vi)).

The sphere is checked against integer brute force (for cells whose |G|^2 is a
rational multiple of an integer form), symmetry, and the lattice-translation
relabelling k -> k + b.  Nothing here re-evaluates the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle
import qeinputs


def _int_sphere_cubic(a, ecut):
    """Integer points with m1^2 + m2^2 + m3^2 <= ecut (a / 2pi)^2 (cubic cell, Gamma)."""
    lim = ecut * (a / (2 * math.pi)) ** 2
    r = int(math.isqrt(int(lim))) + 1
    pts = set()
    for m1 in range(-r, r + 1):
        for m2 in range(-r, r + 1):
            for m3 in range(-r, r + 1):
                if m1 * m1 + m2 * m2 + m3 * m3 <= lim:
                    pts.add((m1, m2, m3))
    return pts


@pytest.mark.parametrize("a,ecut,count", [(10.0, 20.0, 1503), (20.0, 40.0, 34265)])
def test_cubic_sphere_matches_integer_enumeration(a, ecut, count):
    m, kin, _ = oracle.gsphere(qeinputs.cubic(a), np.zeros(3), ecut)
    assert len(m) == count
    assert set(map(tuple, m.tolist())) == _int_sphere_cubic(a, ecut)
    # |G|^2 is (2pi/a)^2 times the integer norm
    n2 = (m ** 2).sum(axis=1)
    np.testing.assert_allclose(kin, (2 * math.pi / a) ** 2 * n2, rtol=1e-14, atol=0)


def test_tetragonal_sphere_integer_form():
    a, c, ecut = 12.0, 24.0, 30.0
    m, _, _ = oracle.gsphere(qeinputs.tetragonal(a, c), np.zeros(3), ecut)
    # |G|^2 = (2pi)^2 (m1^2/a^2 + m2^2/a^2 + m3^2/c^2); c = 2a -> integer form 4m1^2+4m2^2+m3^2
    lim = ecut * (c / (2 * math.pi)) ** 2
    want = set()
    for m1 in range(-12, 13):
        for m2 in range(-12, 13):
            for m3 in range(-25, 26):
                if 4 * m1 * m1 + 4 * m2 * m2 + m3 * m3 <= lim:
                    want.add((m1, m2, m3))
    assert set(map(tuple, m.tolist())) == want
    assert len(m) == 9629


def test_order_ascending_with_lexicographic_ties():
    c = qeinputs.config("SMALL")
    m, kin, _ = oracle.gsphere(c["lat"], c["k"], c["ecut"])
    assert np.all(np.diff(kin) >= 0)
    m0, _, _ = oracle.gsphere(qeinputs.cubic(10.0), np.zeros(3), 20.0)
    # at Gamma in a cubic cell the first shell is the six (+-1,0,0) permutations
    assert tuple(m0[0]) == (0, 0, 0)
    # first shell: 6 vectors, the order within the shell is fixed by the float
    # value then (m1, m2, m3); every member has norm 1
    assert set(map(tuple, m0[1:7].tolist())) == {(-1, 0, 0), (1, 0, 0), (0, -1, 0),
                                                  (0, 1, 0), (0, 0, -1), (0, 0, 1)}


def test_gamma_inversion_symmetry():
    m, _, _ = oracle.gsphere(qeinputs.cubic(10.0), np.zeros(3), 20.0)
    s = set(map(tuple, m.tolist()))
    assert all((-x, -y, -z) in s for x, y, z in s)


def test_k_plus_reciprocal_vector_relabels_the_set():
    c = qeinputs.config("SMALL")
    b = oracle.reciprocal(c["lat"])
    _, kin1, q1 = oracle.gsphere(c["lat"], c["k"], c["ecut"])
    _, kin2, q2 = oracle.gsphere(c["lat"], c["k"] + b[1], c["ecut"])
    assert len(q1) == len(q2)
    a1 = np.array(sorted(map(tuple, np.round(q1, 9).tolist())))
    a2 = np.array(sorted(map(tuple, np.round(q2, 9).tolist())))
    np.testing.assert_allclose(a1, a2, atol=1e-9)


def test_count_close_to_continuum_volume():
    # number of plane waves ~ Omega ecut^{3/2} / (6 pi^2) (volume of the sphere / cell volume in G space)
    for a, ecut in [(10.0, 20.0), (20.0, 40.0), (16.0, 30.0)]:
        m, _, _ = oracle.gsphere(qeinputs.cubic(a), np.zeros(3), ecut)
        est = a ** 3 * ecut ** 1.5 / (6 * math.pi ** 2)
        assert abs(len(m) - est) / est < 0.03


def test_reciprocal_duality():
    lat = np.array([[7.0, 0.3, 0.0], [0.2, 8.0, 0.1], [0.0, -0.4, 9.0]])
    b = oracle.reciprocal(lat)
    np.testing.assert_allclose(lat @ b.T, 2 * math.pi * np.eye(3), atol=1e-13)
    assert abs(oracle.volume(lat) - abs(np.linalg.det(lat))) < 1e-10


def test_grid_check_rejects_wrap():
    m, _, _ = oracle.gsphere(qeinputs.cubic(10.0), np.zeros(3), 20.0)
    oracle.check_grid(m, (15, 15, 15))
    with pytest.raises(ValueError):
        oracle.check_grid(m, (14, 15, 15))
