"""Oracle solve entry point: problem set-up + FGMRES with P_tilde (Sec. 3, Sec. 5).

Test infrastructure only (see the package header).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .aao import AllAtOnce
from .fgmres import fgmres
from .operators import operators, q2_jacobi_interval
from .precond import Preconditioner
from .tableau import tableau


@dataclass
class OracleOptions:
    tol: float = 1e-8
    restart: int = 20
    maxit: int = 100
    inner_maxit: int = 5
    inner_tol: float = 1e-6
    mg_cycles: int = 3
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.8
    cheb_steps: int = 20
    exact: bool = False


@dataclass
class OracleResult:
    x: np.ndarray
    outer_its: int
    rel_res: float
    converged: bool
    inner_its: int
    history: list = field(default_factory=list)


def build(ns, T, nt, method, s, disc="fd", kappa=None, lens=None, tab=None):
    """AllAtOnce operator for the heat problem; tab = (A, b, c) overrides the tableau."""
    M, K = operators(ns, lens, disc, kappa)
    A, b, c = tab if tab is not None else tableau(method, s)
    op = AllAtOnce(K, M, T / nt, nt, A, b, c)
    if disc == "q2":
        op.mass_interval = q2_jacobi_interval(len(ns))
    return op


def solve(op, ns, rhs, opts: OracleOptions, x0=None, transpose=False):
    P = Preconditioner(op, ns, opts.inner_maxit, opts.inner_tol, opts.mg_cycles, opts.nu1,
                       opts.nu2, opts.omega, opts.cheb_steps, opts.exact)
    hist = []
    if transpose:
        x, its, rr, ok = fgmres(op.rmatvec, P.apply_T, rhs, opts.tol, opts.restart, opts.maxit,
                                x0, hist)
    else:
        x, its, rr, ok = fgmres(op.matvec, P.apply, rhs, opts.tol, opts.restart, opts.maxit,
                                x0, hist)
    return OracleResult(x, its, rr, ok, P.inner_its, hist)
