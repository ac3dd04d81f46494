"""Exact all-at-once solve for constant-coefficient finite differences, mode by mode.

Test infrastructure only (see the package header).

With M = I and K = -Delta_h (5-/7-point, zero Dirichlet data, vertex grid,
constant coefficient), K is diagonalised by the orthonormal type-I sine
transform: K = S diag(lambda) S with S = S^T = S^{-1} and, per axis of n
interior points and spacing h, lambda_k = (4 / h^2) sin^2(k pi / (2 (n + 1))),
k = 1..n; in d dimensions the eigenvalues add.  In the sine basis every block of
the all-at-once system of Eq. (system_all_at_once_RK) decouples into one small
system per mode lambda; its rows (Sec. 2) give, for a right-hand side
[r_v ; r_V] transformed blockwise,

  v_0 = r_{v,0};
  (I_s + tau lambda A_RK) V_n = r_{V,n} - lambda v_n e;
  v_{n+1} = v_n + tau sum_i b_i V_{n,i} + r_{v,n+1},

i.e. the forward substitution of oracle.sequential with Theta_hat replaced by
its s x s restriction to the mode (invertible: the eigenvalues of A_RK have
positive real part for Radau IIA and Gauss, lambda > 0).  The result is the
exact solution of the all-at-once system up to rounding, at any size the
memory holds (the cost per time step is 2(s + 1) sine transforms).

Pins (tests): equal to oracle.sequential.sequential_solve (sparse LU of
Theta_hat) on 2D and 3D grids with Radau IIA and Gauss tableaus; the
eigenvalues against a dense eigendecomposition of K; the unforced sine
eigenmode propagated by R(-tau lambda)^n.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def _shape(ns):
    """Array shape of a flattened grid vector (x fastest)."""
    return tuple(reversed(tuple(int(n) for n in ns)))


def eigenvalues(ns, lens=None):
    """Eigenvalues of K = -Delta_h on the vertex grid, in the layout of the sine transform."""
    ns = tuple(int(n) for n in ns)
    lens = tuple(lens) if lens is not None else (1.0,) * len(ns)
    lam = np.zeros(_shape(ns))
    d = len(ns)
    for a, (n, L) in enumerate(zip(ns, lens)):
        h = L / (n + 1)
        k = np.arange(1, n + 1)
        la = (4.0 / (h * h)) * np.sin(k * np.pi / (2.0 * (n + 1))) ** 2
        shape = [1] * d
        shape[d - 1 - a] = n          # axis a (x = 0) is the last array axis
        lam = lam + la.reshape(shape)
    return lam.reshape(-1)


def sine(v, ns):
    """Orthonormal type-I sine transform of a grid vector (its own inverse)."""
    return sfft.dstn(np.asarray(v, dtype=np.float64).reshape(_shape(ns)), type=1, norm="ortho").reshape(-1)


def solve(ns, tau, nt, A, b, rhs, lens=None):
    """x = A_aao^{-1} rhs for the FD all-at-once operator with M = I, K = -Delta_h (constant
    coefficient), tableau (A, b), nt steps of size tau; rhs and x in the paper's ordering
    [v_0 .. v_nt ; V_0 .. V_{nt-1}]."""
    A = np.asarray(A, dtype=np.float64)
    bw = np.asarray(b, dtype=np.float64)
    s = len(bw)
    lam = eigenvalues(ns, lens)
    nx = lam.size
    rhs = np.asarray(rhs, dtype=np.float64)
    nv = (nt + 1) * nx
    rv = rhs[:nv].reshape(nt + 1, nx)
    rV = rhs[nv:].reshape(nt, s, nx)
    # per-mode stage matrices (I + tau lambda A)^{-1}, shape (nx, s, s)
    G = np.linalg.inv(np.eye(s)[None, :, :] + tau * lam[:, None, None] * A[None, :, :])
    v = np.empty((nt + 1, nx))
    V = np.empty((nt, s, nx))
    vh = sine(rv[0], ns)
    v[0] = sine(vh, ns)
    for n in range(nt):
        rhat = np.stack([sine(rV[n, i], ns) for i in range(s)], axis=1)     # (nx, s)
        rhat = rhat - lam[:, None] * vh[:, None]
        Vh = np.einsum("pij,pj->pi", G, rhat)                               # (nx, s)
        for i in range(s):
            V[n, i] = sine(Vh[:, i], ns)
        vh = vh + tau * (Vh @ bw) + sine(rv[n + 1], ns)
        v[n + 1] = sine(vh, ns)
    return np.concatenate([v.reshape(-1), V.reshape(-1)])
