"""Adjoint solve and gradients of a tracking functional (test infrastructure only).

For 𝒜(kappa) x = rhs(f, u0) (Eq. system_all_at_once_RK) and a functional J(x, f),
dJ/dtheta = lambda^T (d rhs/d theta - (d𝒜/d theta) x) + dJ/dtheta|_explicit with
𝒜^T lambda = dJ/dx.  For the source f (constant in time, rhs_{V,n,i} = M f) and the
nodal diffusivity kappa (K depends on kappa through face averages,
kappa_f = (kappa_P + kappa_Q)/2):

  dJ/df      = sum_{n,i} M^T lambda_{V,n,i}
  dJ/du0     = M^T lambda_{v,0}
  dJ/dkappa_m = - sum_{n,i} sum_{faces f = (P,Q) touching node m} (1/2) h_f^{-2}
                  (lambda_{V,n,i,P} - lambda_{V,n,i,Q}) (W_{n,i,P} - W_{n,i,Q}),
  W_{n,i} = v_n + tau sum_j a_ij V_{n,j}   (the argument of K in (𝒜 x)_{V,n,i}),
with boundary values 0.  The tracking functional of the gradient workload is
J = 1/2 ||v_nt - u_target||^2 + 1/2 * 1e-4 ||f||^2.

Pins (tests): gradients against central finite differences of J with dense LU
solves on tiny grids; the adjoint solution against a dense transposed solve.
"""
from __future__ import annotations

import numpy as np

from .fgmres import fgmres
from .precond import Preconditioner


def tracking_dJdx(op, x, target):
    """dJ/dx for J = 1/2 ||v_nt - target||^2: nonzero only in the v_nt block."""
    g = np.zeros(op.n_st)
    lo = op.nt * op.nx
    g[lo: lo + op.nx] = x[lo: lo + op.nx] - target
    return g


def tracking_J(op, x, f, target, reg=1e-4):
    lo = op.nt * op.nx
    d = x[lo: lo + op.nx] - target
    return 0.5 * d @ d + 0.5 * reg * f @ f


def adjoint_solve(op, ns, dJdx, tol=1e-12, restart=20, maxit=100, **pkw):
    P = Preconditioner(op, ns, **pkw)
    lam, its, rr, ok = fgmres(op.rmatvec, P.apply_T, dJdx, tol, restart, maxit)
    return lam, its, rr, ok


def grad_f(op, lam):
    _, lV = op.split(lam)
    acc = np.zeros(op.nx)
    for n in range(op.nt):
        for i in range(op.s):
            acc = acc + op.MTmul(lV[n, i])
    return acc


def grad_u0(op, lam):
    lv, _ = op.split(lam)
    return op.MTmul(lv[0])


def grad_kappa(op, ns, lam, x, lens=None):
    """Face-by-face accumulation over all (N+2)^d nodes (FD only)."""
    ns = tuple(ns)
    d = len(ns)
    lens = lens if lens is not None else (1.0,) * d
    h2 = [((n + 1) / L) ** 2 for n, L in zip(ns, lens)]
    v, V = op.split(x)
    _, lV = op.split(lam)
    full = tuple(n + 2 for n in ns[::-1])                # array shape, x last
    grad = np.zeros(full)
    inner = tuple(slice(1, n + 1) for n in ns[::-1])
    for n in range(op.nt):
        for i in range(op.s):
            W = v[n].copy()
            for j in range(op.s):
                W = W + op.tau * op.A[i, j] * V[n, j]
            Wf = np.zeros(full)
            Lf = np.zeros(full)
            Wf[inner] = W.reshape(ns[::-1])
            Lf[inner] = lV[n, i].reshape(ns[::-1])
            for a in range(d):
                ax = d - 1 - a
                lo = [slice(None)] * d
                hi = [slice(None)] * d
                lo[ax] = slice(0, full[ax] - 1)
                hi[ax] = slice(1, full[ax])
                prod = 0.5 * h2[a] * (Lf[tuple(lo)] - Lf[tuple(hi)]) * (Wf[tuple(lo)] - Wf[tuple(hi)])
                # faces between two boundary nodes carry zero differences already
                grad[tuple(lo)] -= prod
                grad[tuple(hi)] -= prod
    return grad.reshape(-1)
