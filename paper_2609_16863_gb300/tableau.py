"""Butcher tableaus for the solver's aao_tableau argument (Sec. 2).

Radau IIA nodes: c_s = 1 and c_1..c_{s-1} = (1 + x_i)/2 with x_i the zeros of
the Jacobi polynomial P_{s-1}^{(1,0)}; Gauss--Legendre nodes: (1 + x_i)/2 with
x_i the Gauss points.  For both collocation families A and b follow from the
simplifying conditions C(s) and B(s):
    sum_j a_ij c_j^{k-1} = c_i^k / k,   sum_j b_j c_j^{k-1} = 1/k,   k = 1..s,
i.e. A = C V^{-1}, b = q V^{-1} with the Vandermonde matrix V_{kj} = c_j^{k-1}.
"""
from __future__ import annotations

import numpy as np
from scipy.special import roots_jacobi


def _from_nodes(c: np.ndarray):
    s = len(c)
    k = np.arange(1, s + 1)
    V = c[None, :] ** (k[:, None] - 1)                   # V[k-1, j] = c_j^{k-1}
    Cm = c[:, None] ** k[None, :] / k[None, :]           # Cm[i, k-1] = c_i^k / k
    A = np.linalg.solve(V, Cm.T).T                       # A V^T = Cm
    b = np.linalg.solve(V, 1.0 / k)
    return A, b, c


def radau_iia(s: int):
    if s == 1:
        return _from_nodes(np.array([1.0]))
    x, _ = roots_jacobi(s - 1, 1.0, 0.0)
    c = np.concatenate([np.sort((1.0 + x) / 2.0), [1.0]])
    return _from_nodes(c)


def gauss_legendre(s: int):
    x, _ = np.polynomial.legendre.leggauss(s)
    return _from_nodes(np.sort((1.0 + x) / 2.0))


def make(method: str, s: int):
    if method == "radau":
        return radau_iia(s)
    if method == "gauss":
        return gauss_legendre(s)
    raise ValueError(f"unknown RK family {method!r}")
