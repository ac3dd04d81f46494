"""Restarted right-preconditioned flexible GMRES (Algorithm 1, P_L = I).

Test infrastructure only (see the package header).

Algorithm 1 with u = u_A = FP64, P_L = I and P_R = P_tilde; modified
Gram--Schmidt Arnoldi, Givens rotations for the least-squares problem, the
preconditioned directions z_k kept (flexible variant, needed because
P_tilde contains GMRES and is not a fixed linear map, Sec. 3).

Restart and stopping (Sec. 5: restart 20, tolerance 1e-8 on the relative
residual, at most 100 iterations).  With b the right-hand side:
  r = b - A x, beta = ||r||;
  a cycle stops at iteration k when |g_{k+1}| <= tol ||b||, or h_{k+1,k} = 0,
  or the cycle has `restart` iterations, or `maxit` iterations were used;
  then x <- x + Z_k y_k and the true residual is recomputed;
  the solve has converged when the TRUE residual satisfies
  ||b - A x|| <= tol ||b||.

Pins (tests): solutions against dense LU of the assembled operator (2D/3D,
s = 1..3, Radau and Gauss); the exact-inverse preconditioner converging in
two iterations (minimal polynomial of degree 2, Sec. 3).
"""
from __future__ import annotations

import numpy as np

from .precond import givens


def fgmres(apply_A, apply_P, b, tol=1e-8, restart=20, maxit=100, x0=None, history=None):
    """Returns (x, outer_iterations, true_relative_residual, converged)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    r = b - apply_A(x) if x0 is not None else b.copy()
    beta = float(np.linalg.norm(r))
    total = 0
    m = int(restart)
    while True:
        if beta <= tol * bnorm:
            return x, total, beta / bnorm, True
        if total >= maxit:
            return x, total, beta / bnorm, False
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k_used = 0
        for k in range(m):
            total += 1
            Z.append(apply_P(V[k]))
            w = apply_A(Z[k])
            for i in range(k + 1):
                H[i, k] = float(V[i] @ w)
                w = w - H[i, k] * V[i]
            hk1 = float(np.linalg.norm(w))
            H[k + 1, k] = hk1
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            cs[k], sn[k], H[k, k] = givens(H[k, k], hk1)
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            if history is not None:
                history.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) <= tol * bnorm or hk1 == 0.0 or total >= maxit:
                break
            if k < m - 1:
                V.append(w / hk1)
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:k_used]) / H[i, i]
        for i in range(k_used):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
