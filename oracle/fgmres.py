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

fgmres_split is Algorithm 1 with a left preconditioner as well (the paper's
parallel runs precondition on the left).  Pins: P_L = I reproduces fgmres
iterate for iterate; the exact P_tilde converges in two iterations on either
side; P_L = A^{-1} in one; a left-preconditioned solve with the inexact
P_tilde against a dense solve.
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


def fgmres_split(apply_A, apply_PL, apply_PR, b, tol=1e-8, restart=20, maxit=100, x0=None, history=None):
    """Algorithm 1: FGMRES with split preconditioning, P_L applied on the left of A and P_R (which
    may change from one iteration to the next) on the right, in FP64.

    Per Algorithm 1: t = A x_0, r_0 = P_L^{-1} b - P_L^{-1} t, beta = ||r_0||, v_1 = r_0 / beta;
    iteration k: z_k = P_R^{-1} v_k, w = P_L^{-1} (A z_k), modified Gram--Schmidt against
    v_1..v_k, h_{k+1,k} = ||w||, y_k = argmin ||beta e_1 - H_k y|| (Givens rotations); x = x_0 +
    Z_k y_k.  Reading for the restarted form used in Sec. 5 (restart 20 / 15): a cycle ends when
    ||beta e_1 - H_k y_k|| <= tol beta_0 (Algorithm 1's test, beta_0 the first cycle's beta) or
    after `restart` iterations; the next cycle restarts from the iterate; the solve has converged
    when the recomputed ||P_L^{-1} b - P_L^{-1} A x|| <= tol beta_0.  With P_L = I this is the
    right-preconditioned `fgmres` above, iterate for iterate.
    Returns (x, iterations, true relative residual ||b - A x|| / ||b||, converged)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    bt = apply_PL(b)
    beta0 = None
    total = 0
    m = int(restart)
    while True:
        r = bt - apply_PL(apply_A(x))
        beta = float(np.linalg.norm(r))
        if beta0 is None:
            beta0 = beta
        if beta <= tol * beta0 or total >= maxit:
            rt = float(np.linalg.norm(b - apply_A(x))) / bnorm
            return x, total, rt, beta <= tol * beta0
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
            Z.append(apply_PR(V[k]))
            w = apply_PL(apply_A(Z[k]))
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
                history.append(abs(g[k + 1]) / beta0)
            if abs(g[k + 1]) <= tol * beta0 or hk1 == 0.0 or total >= maxit:
                break
            if k < m - 1:
                V.append(w / hk1)
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:k_used]) / H[i, i]
        for i in range(k_used):
            x = x + y[i] * Z[i]
