"""Pins of the oracle's 1D tables against closed forms and an independent library routine.

Paper: Sec. 3.1 (nodal Gauss-Lobatto basis, sum factorisation over 1D tables).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg


@pytest.mark.parametrize("k,expected", [
    (1, [0.0, 1.0]),
    (2, [0.0, 0.5, 1.0]),
    (3, [0.0, (1 - 1 / math.sqrt(5)) / 2, (1 + 1 / math.sqrt(5)) / 2, 1.0]),
    (4, [0.0, (1 - math.sqrt(3 / 7)) / 2, 0.5, (1 + math.sqrt(3 / 7)) / 2, 1.0]),
])
def test_gll_closed_forms(oracle, k, expected):
    np.testing.assert_allclose(oracle.gll_nodes(k), expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", range(1, 9))
def test_gll_interior_are_roots_of_dPk(oracle, k):
    # independent: numpy's Legendre series derivative roots
    r = np.sort(npleg.Legendre.basis(k).deriv().roots().real) if k > 1 else np.array([])
    ref = np.concatenate([[0.0], (r + 1) / 2, [1.0]])
    np.testing.assert_allclose(oracle.gll_nodes(k), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_matches_numpy_leggauss(oracle, n):
    x, w = oracle.gauss(n)
    xr, wr = npleg.leggauss(n)
    np.testing.assert_allclose(x, (xr + 1) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wr / 2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exactness(oracle, n):
    x, w = oracle.gauss(n)
    for m in range(2 * n):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) < 5e-15
    # one degree higher the error is the classical remainder (n!)^4 / ((2n+1) ((2n)!)^2)
    err = 1.0 / (2 * n + 1) - np.dot(w, x ** (2 * n))
    ref = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs(err - ref) < 0.01 * ref + 5e-15


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_properties(oracle, k):
    nodes = oracle.gll_nodes(k)
    for j, s in enumerate(nodes):
        phi, _ = oracle.lagrange(nodes, s)
        np.testing.assert_allclose(phi, np.eye(k + 1)[j], atol=1e-14)
    for s in np.linspace(0.0, 1.0, 13):
        phi, dphi = oracle.lagrange(nodes, s)
        assert abs(phi.sum() - 1.0) < 1e-13
        assert abs(dphi.sum()) < 1e-11
        # interpolant of s^m (m <= k) is exact, and so is its derivative
        for m in range(k + 1):
            assert abs(np.dot(phi, nodes ** m) - s ** m) < 1e-13
            dm = m * s ** (m - 1) if m > 0 else 0.0
            assert abs(np.dot(dphi, nodes ** m) - dm) < 1e-11


def test_lagrange_derivative_finite_difference(oracle):
    nodes = oracle.gll_nodes(5)
    s, h = 0.37, 1e-6
    _, d = oracle.lagrange(nodes, s)
    p1, _ = oracle.lagrange(nodes, s + h)
    p0, _ = oracle.lagrange(nodes, s - h)
    np.testing.assert_allclose(d, (p1 - p0) / (2 * h), atol=1e-6)
