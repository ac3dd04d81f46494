"""Butcher tableaus by collocation, RK stability function, LDU of A_RK.

Test infrastructure only (see the package header).

Sec. 2 defines an s-stage RK method by its tableau (c_RK | A_RK ; b_RK^T).
Radau IIA and Gauss--Legendre are collocation methods: the nodes c are the
zeros of P_s(2x-1) - P_{s-1}(2x-1) (Radau IIA, right end point included) or of
P_s(2x-1) (Gauss), and a_ij = int_0^{c_i} l_j(t) dt, b_j = int_0^1 l_j(t) dt
with l_j the Lagrange basis on the nodes.

Pins (tests): row sums of A equal c; Radau IIA has b = last row of A;
quadrature order conditions sum_j b_j c_j^{k-1} = 1/k up to k = 2s-1 (Radau)
or 2s (Gauss); the stability function equals the Pade closed forms; L D U
reconstructs A.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def _shifted_legendre(k: int) -> np.ndarray:
    """Power-series coefficients of P_k(2x - 1)."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    p = npleg.leg2poly(c)                    # in t
    # substitute t = 2x - 1
    out = np.zeros(1)
    tpow = np.array([1.0])
    for a in p:
        out = nppoly.polyadd(out, a * tpow)
        tpow = nppoly.polymul(tpow, [-1.0, 2.0])
    return out


def _collocation(c: np.ndarray):
    s = len(c)
    A = np.zeros((s, s))
    b = np.zeros(s)
    for j in range(s):
        lj = np.array([1.0])
        for m in range(s):
            if m != j:
                lj = nppoly.polymul(lj, np.array([-c[m], 1.0]) / (c[j] - c[m]))
        Lj = nppoly.polyint(lj)
        for i in range(s):
            A[i, j] = nppoly.polyval(c[i], Lj)
        b[j] = nppoly.polyval(1.0, Lj)
    return A, b


def radau_iia(s: int):
    """Radau IIA tableau (A, b, c), s >= 1."""
    if s == 1:
        c = np.array([1.0])
    else:
        poly = nppoly.polysub(_shifted_legendre(s), _shifted_legendre(s - 1))
        r = np.sort(np.real(nppoly.polyroots(poly)))
        r[-1] = 1.0
        c = r
    A, b = _collocation(c)
    return A, b, c


def gauss_legendre(s: int):
    """Gauss--Legendre tableau (A, b, c), s >= 1."""
    c = np.sort(np.real(nppoly.polyroots(_shifted_legendre(s))))
    A, b = _collocation(c)
    return A, b, c


def tableau(method: str, s: int):
    if method == "radau":
        return radau_iia(s)
    if method == "gauss":
        return gauss_legendre(s)
    raise ValueError(method)


def stability_function(A: np.ndarray, b: np.ndarray, z: complex) -> complex:
    """R(z) = 1 + z b^T (I - z A)^{-1} e."""
    s = len(b)
    e = np.ones(s)
    return 1.0 + z * (b @ np.linalg.solve(np.eye(s) - z * A, e))


def ldu(A: np.ndarray):
    """A = L D U without pivoting; L unit lower, D diagonal, U unit upper."""
    s = A.shape[0]
    L = np.eye(s)
    U = np.eye(s)
    D = np.zeros(s)
    W = A.astype(float).copy()
    for k in range(s):
        D[k] = W[k, k]
        if D[k] == 0.0:
            raise ZeroDivisionError("zero pivot in LDU of A_RK")
        for i in range(k + 1, s):
            L[i, k] = W[i, k] / D[k]
        for j in range(k + 1, s):
            U[k, j] = W[k, j] / D[k]
        for i in range(k + 1, s):
            for j in range(k + 1, s):
                W[i, j] -= L[i, k] * D[k] * U[k, j]
    return L, D, U
