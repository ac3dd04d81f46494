"""Pins of the oracle's Butcher tableaus, stability functions and LDU (Sec. 2, Sec. 3)."""
import math

import numpy as np
import pytest

from oracle.tableau import gauss_legendre, ldu, radau_iia, stability_function

# Pade closed forms of the stability functions (Hairer & Wanner, Solving ODEs II,
# Table IV.5.x): Radau IIA s is the (s-1, s) subdiagonal Pade approximant of e^z,
# Gauss s the (s, s) diagonal one.
PADE = {
    ("radau", 1): lambda z: 1.0 / (1.0 - z),
    ("radau", 2): lambda z: (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6),
    ("radau", 3): lambda z: (1 + 2 * z / 5 + z * z / 20) / (1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60),
    ("gauss", 1): lambda z: (1 + z / 2) / (1 - z / 2),
    ("gauss", 2): lambda z: (1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12),
}


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_radau_structure(s):
    A, b, c = radau_iia(s)
    assert np.allclose(A.sum(axis=1), c, atol=1e-14)
    assert np.allclose(b, A[-1], atol=1e-14)      # stiffly accurate
    assert abs(c[-1] - 1.0) < 1e-15
    # quadrature order 2s-1
    for k in range(1, 2 * s):
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13
    assert abs(b @ c ** (2 * s - 1) - 1.0 / (2 * s)) > 1e-6   # and not higher


@pytest.mark.parametrize("s", [1, 2, 3])
def test_gauss_structure(s):
    A, b, c = gauss_legendre(s)
    assert np.allclose(A.sum(axis=1), c, atol=1e-14)
    for k in range(1, 2 * s + 1):
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13


def test_textbook_values():
    # Radau IIA s=2 and Gauss s=2 in closed form (Hairer & Wanner, Table IV.5.5/5.1)
    A, b, c = radau_iia(2)
    assert np.allclose(A, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)
    assert np.allclose(c, [1 / 3, 1], atol=1e-15)
    A, b, c = gauss_legendre(2)
    r = math.sqrt(3) / 6
    assert np.allclose(A, [[1 / 4, 1 / 4 - r], [1 / 4 + r, 1 / 4]], atol=1e-15)
    assert np.allclose(c, [0.5 - r, 0.5 + r], atol=1e-15)
    A, b, c = radau_iia(3)
    s6 = math.sqrt(6)
    assert np.allclose(c, [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)
    assert np.allclose(A[0], [(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225], atol=1e-14)


@pytest.mark.parametrize("key", list(PADE))
def test_stability_function_pade(key):
    method, s = key
    A, b, c = (radau_iia if method == "radau" else gauss_legendre)(s)
    for z in (-0.3, -2.0, -17.5, -1e3, 0.4 + 0.7j):
        R = stability_function(A, b, z)
        assert abs(R - PADE[key](z)) <= 1e-12 * max(1.0, abs(R))


@pytest.mark.parametrize("maker,s", [(radau_iia, 2), (radau_iia, 3), (radau_iia, 5), (gauss_legendre, 2)])
def test_ldu_reconstructs(maker, s):
    A, _, _ = maker(s)
    L, D, U = ldu(A)
    assert np.allclose(L @ np.diag(D) @ U, A, atol=1e-15)
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
    assert np.allclose(np.tril(U, -1), 0) and np.allclose(np.diag(U), 1)
    assert np.all(D > 0)   # every shifted block M + tau d_i K is SPD


def test_ldu_pivots_radau2():
    _, D, _ = ldu(radau_iia(2)[0])
    # d1 = a11 = 5/12, d2 = det(A)/a11 = (5/48 + 3/48) / (5/12) = 2/5
    assert np.allclose(D, [5 / 12, 2 / 5], atol=1e-15)
