"""Relaxed (iteration-dependent) matvec precision in FGMRES: the future-work direction of the
paper's introduction, after the inexact-Krylov theory it cites (Simoncini and Szyld).

Test infrastructure only (see the package header).

Right-preconditioned FGMRES (Algorithm 1 with P_L = I) in which iteration k of a cycle may form
w = A z_k with a cheaper, inexact product w = A z_k + f_k.  With y the cycle's least-squares
coefficients, the computed residual r~ = beta e_1 - H y and the true residual of x = x_0 + Z y
differ by F y = sum_k f_k y_k, and |y_k| <= ||r~_{k-1}|| / sigma_min(H_bar) (Simoncini and Szyld,
Lemma 5.1, for any Hessenberg least-squares problem of this form).  So if every inexact product
satisfies

    ||f_k|| <= allowed_k = ell * tol * ||b|| / (m * ||r~_{k-1}||)           (m = restart)

the gap after j iterations is at most ell * tol * ||b|| * (j / m) / sigma_min(H_bar): the
tolerance on a product grows as the residual falls.  Reading (the paper gives no rule): the
inexact product is tried at every iteration and accepted when its a-posteriori error bound is
within allowed_k, else A z_k is recomputed exactly; ||r~_{k-1}|| is |g_k|, the current Givens
residual; a cycle ends and the solve converges exactly as in `fgmres`, on the TRUE residual
recomputed with the exact product, so the relaxation never changes the stopping test.

`fp32_product` is one inexact product: z and the operator's entries rounded to FP32 and every
product and sum in FP32, with the rigorous componentwise bound |fl(A z) - A z| <= gamma_d |A| |z|
(Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1: every entry of the result is
a sum of products, and d bounds the number of roundings on any path from an input to the
result), reported in the 2-norm.

Pins (tests/test_oracle_relaxed.py): ell = 0 and an exact product both reproduce `fgmres`
iterate for iterate; with a worst-case inexact product (error of exactly the allowed norm in a
random direction) the computed-vs-true residual gap obeys the bound above; the FP32 product obeys
its componentwise bound against the exact product and the bound is not vacuous (within a factor
of the observed error on a cancellation-free operator); a relaxed solve of the all-at-once system
reaches the tolerance on its true residual with P_tilde as the preconditioner.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .precond import givens

U32 = 2.0 ** -24          # unit roundoff of FP32 (round to nearest)


def gamma(d: int, u: float = U32) -> float:
    """gamma_d = d u / (1 - d u) (Higham Sec. 3.1)."""
    return d * u / (1.0 - d * u)


def fp32_product(A: sp.csr_matrix, z: np.ndarray, depth: int | None = None):
    """(w, bound): w = A z with z and A's entries rounded to FP32 and FP32 arithmetic, returned in
    FP64; bound = gamma_d || |A| |z| ||_2 >= ||w - A z||_2.  For a CSR row of nnz terms the path
    from an input to the result holds the rounding of the entry, of the input, of the product and
    at most nnz - 1 additions: d = nnz_max + 2 unless `depth` is given."""
    A = sp.csr_matrix(A)
    A32 = A.astype(np.float32)
    w = (A32 @ np.asarray(z, dtype=np.float64).astype(np.float32)).astype(np.float64)
    if depth is None:
        depth = int(np.diff(A.indptr).max()) + 2
    absAz = abs(A) @ np.abs(np.asarray(z, dtype=np.float64))
    return w, gamma(depth) * float(np.linalg.norm(absAz))


def fgmres_relaxed(apply_A, apply_A_low, apply_P, b, tol=1e-8, restart=20, maxit=100, ell=1.0, x0=None,
                   history=None, log=None):
    """FGMRES as oracle.fgmres.fgmres with the relaxed product.  apply_A_low(z, allowed) returns
    (w_low, bound) with ||w_low - A z|| <= bound (it may use `allowed` to pick its accuracy).
    `log` (a list) receives one dict per iteration: allowed, bound, relaxed (the inexact product
    was used); and at the end of each cycle the cycle's gap |r_true - |g||, sigma_min of its
    triangular factor and its coefficients y.
    Returns (x, outer_iterations, true_relative_residual, converged)."""
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
            allowed = ell * tol * bnorm / (m * abs(g[k]))
            w_low, bound = apply_A_low(Z[k], allowed)
            relaxed = bound <= allowed
            w = w_low if relaxed else apply_A(Z[k])
            if log is not None:
                log.append({"allowed": allowed, "bound": bound, "relaxed": bool(relaxed)})
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
        if log is not None:
            smin = float(np.linalg.svd(H[:k_used, :k_used], compute_uv=False).min())
            log.append({"cycle_end": True, "iterations": k_used, "gap": abs(beta - abs(g[k_used])),
                        "sigma_min": smin, "y": y.copy()})
