"""Python front end of the C ABI: one `Solver` per heat problem.

Vectors are torch float64 tensors on the GPU (used in place, on the solver's
stream) or float64 numpy arrays on the host (the library copies them through
its workspace).  Every operation runs in libaao_rk.so; this module only
marshals arguments.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import _lib
from .tableau import make as make_tableau


def _ptr(a, n=None, what="vector"):
    """Address of a contiguous float64 torch tensor or numpy array (None -> NULL).  With n given
    the vector must hold at least n values: the library reads or writes exactly n values through
    the address and cannot check the length itself."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy vectors must be contiguous float64")
        size, addr = a.size, a.ctypes.data
    else:
        import torch
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"unsupported vector type {type(a)}")
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch vectors must be contiguous float64")
        size, addr = a.numel(), a.data_ptr()
    if n is not None and size < n:
        raise ValueError(f"{what} holds {size} values, {n} are needed")
    return addr


@dataclass
class Info:
    outer_its: int
    inner_its_total: int
    rel_res: float
    converged: bool
    t_theta_ms: float
    t_schur_ms: float
    t_total_ms: float
    history: list = field(default_factory=list)
    relaxed_matvecs: int = 0

    @staticmethod
    def from_c(ci: _lib.aao_info) -> "Info":
        return Info(ci.outer_its, ci.inner_its_total, ci.rel_res, bool(ci.converged), ci.t_theta_ms,
                    ci.t_schur_ms, ci.t_total_ms, [ci.history[i] for i in range(ci.n_history)],
                    ci.relaxed_matvecs)


class Solver:
    """Handle for one problem: grid n (interior points per axis), final time T,
    nt steps, an RK tableau (A, b, c), optional nodal diffusivity kappa.  mgrit_m in 2..nt
    replaces S_tilde's forward substitution by one two-level MGRIT iteration with coarsening
    factor mgrit_m (C-points at its multiples; a shorter final interval where it does not
    divide nt; tune.tune_mgrit picks one by timing); precond_side="left" runs Algorithm 1 with
    P_L = P_tilde, P_R = I instead of the right-preconditioned FGMRES.  relax_matvec = ell > 0
    lets late outer iterations keep an FP32 product A z_k whose error bound is within the
    inexact-Krylov allowance ell tol ||b|| / (restart |g_k|) (aao_options.relax_matvec)."""

    def __init__(self, n: Sequence[int], T: float, nt: int, tableau=None, method: str = "radau", s: int = 2,
                 lens=None, kappa=None, prec_P: str = "fp64", prec_Pint: Optional[str] = None,
                 tol: float = 1e-8, restart: int = 20, maxit: int = 100, inner_maxit: int = 0,
                 inner_tol: float = -1.0, mg_cycles: int = 3, mg_pre: int = 2, mg_post: int = 2,
                 mg_omega: float = 0.8, disc: str = "fd", cheb_steps: int = 20, stream=None, mgrit_m: int = 0,
                 precond_side: str = "right", relax_matvec: float = 0.0):
        self._lib = _lib.lib()
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.n_nodes = int(np.prod([v + 2 for v in self.n]))    # nodal kappa, boundary included
        A, b, c = tableau if tableau is not None else make_tableau(method, s)
        A, b, c = np.asarray(A, float), np.asarray(b, float), np.asarray(c, float)
        self.s = len(b)
        self.nt = int(nt)
        self.tau = float(T) / self.nt
        g = _lib.aao_grid()
        g.dim = self.dim
        for a in range(3):
            g.n[a] = self.n[a] if a < self.dim else 1
            g.len[a] = (lens[a] if lens is not None else 1.0) if a < self.dim else 1.0
        g.disc = _lib.DISC[disc]
        self._kappa = kappa     # keep alive until set-up copied it
        g.kappa = _ptr(kappa, self.n_nodes, "kappa")
        t = _lib.aao_tableau()
        t.s = self.s
        for i in range(self.s):
            for j in range(self.s):
                t.A[i * self.s + j] = A[i, j]
            t.b[i] = b[i]
            t.c[i] = c[i]
        o = _lib.aao_options()
        self._lib.aao_rk_default_options(C.byref(o))
        o.tol, o.restart, o.maxit = tol, restart, maxit
        o.inner_maxit, o.inner_tol = inner_maxit, inner_tol
        o.mg_cycles, o.mg_pre, o.mg_post, o.mg_omega = mg_cycles, mg_pre, mg_post, mg_omega
        o.cheb_steps = cheb_steps
        o.prec_P = _lib.PREC[prec_P]
        o.prec_Pint = _lib.PREC[prec_Pint if prec_Pint is not None else prec_P]
        o.stream = stream
        o.mgrit_m = mgrit_m
        o.precond_side = {"right": 0, "left": 1}[precond_side]
        o.relax_matvec = relax_matvec
        self.options = o
        h = C.c_void_p()
        _lib.check(self._lib.aao_rk_setup(C.byref(g), self.tau, self.nt, C.byref(t), C.byref(o), C.byref(h)))
        self.h = h
        nx, nst = C.c_longlong(), C.c_longlong()
        _lib.check(self._lib.aao_rk_sizes(h, C.byref(nx), C.byref(nst)))
        self.nx, self.n_st = nx.value, nst.value
        self.n_v = (self.nt + 1) * self.nx

    def _n_f(self, f_time_dep):
        """Length of a source: one spatial field, or one per stage and time step."""
        return self.nt * self.s * self.nx if f_time_dep else self.nx

    def close(self):
        if getattr(self, "h", None):
            self._lib.aao_rk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operator and preconditioner --------------------------------------------
    def set_tolerances(self, tol=None, maxit=None, inner_tol=None, restart=None):
        o = self.options
        if tol is not None:
            o.tol = tol
        if maxit is not None:
            o.maxit = maxit
        if inner_tol is not None:
            o.inner_tol = inner_tol
        if restart is not None:
            o.restart = restart
        _lib.check(self._lib.aao_rk_set_options(self.h, C.byref(o)))

    def rhs(self, f, u0, out, f_time_dep=False):
        """out (n_st) = the all-at-once right-hand side [M u0 ; 0 ; M f at every stage] for the source f
        (n_x values, or nt*s*n_x at the stage times with f_time_dep) and initial data u0 (n_x)."""
        _lib.check(self._lib.aao_rk_rhs(self.h, _ptr(f, self._n_f(f_time_dep), "f"), int(f_time_dep),
                                        _ptr(u0, self.nx, "u0"), _ptr(out, self.n_st, "out")))
        return out

    def matvec(self, x, y, transpose=False):
        """y = A x (or A^T x), FP64, n_st values each."""
        fn = self._lib.aao_rk_matvec_transpose if transpose else self._lib.aao_rk_matvec
        _lib.check(fn(self.h, _ptr(x, self.n_st, "x"), _ptr(y, self.n_st, "y")))
        return y

    def matvec_relaxed(self, x, y, absy, transpose=False):
        """y = fl32(A x) (or A^T x) and absy = its absolute expression, with |y - A x| <= gamma_32
        absy entry by entry (the relaxed outer product); device arrays of n_st values."""
        _lib.check(self._lib.aao_rk_matvec_relaxed(self.h, _ptr(x, self.n_st, "x"), _ptr(y, self.n_st, "y"),
                                                   _ptr(absy, self.n_st, "absy"), int(bool(transpose))))
        return y, absy

    def precond_apply(self, r, z, transpose=False):
        """z = P_tilde^{-1} r (or P_tilde^{-T} r), n_st values each."""
        fn = self._lib.aao_rk_precond_apply_transpose if transpose else self._lib.aao_rk_precond_apply
        _lib.check(fn(self.h, _ptr(r, self.n_st, "r"), _ptr(z, self.n_st, "z")))
        return z

    def shifted_solve(self, stage, b, x):
        """x ~= (M + tau d_stage K)^{-1} b by the multigrid V-cycles (n_x values each)."""
        _lib.check(self._lib.aao_rk_shifted_solve(self.h, int(stage), _ptr(b, self.nx, "b"),
                                                  _ptr(x, self.nx, "x")))
        return x

    def pint_apply(self, r, y, transpose=False):
        """y = P_int^{-1} r (or P_int^{-T} r) for one time step, s*n_x values each."""
        n = self.s * self.nx
        _lib.check(self._lib.aao_rk_pint_apply(self.h, _ptr(r, n, "r"), _ptr(y, n, "y"), int(transpose)))
        return y

    def inner_solve(self, nblocks, r, z):
        """z_n = Theta_tilde^{-1} r_n for nblocks time blocks of s*n_x values; returns (z, iterations)."""
        its = (C.c_int * nblocks)()
        n = int(nblocks) * self.s * self.nx
        _lib.check(self._lib.aao_rk_inner_solve(self.h, int(nblocks), _ptr(r, n, "r"), _ptr(z, n, "z"), its))
        return z, list(its)

    # -- solves ---------------------------------------------------------------------
    def solve(self, f, u0, x, x0_given=False, f_time_dep=False, allow_not_converged=False):
        """Solve A x = rhs(f, u0) by FGMRES with P_tilde; x (n_st) is the initial guess with x0_given.
        Returns (x, Info); raises AaoError on failure (not on non-convergence with allow_not_converged)."""
        info = _lib.aao_info()
        _lib.check(self._lib.aao_rk_solve(self.h, _ptr(f, self._n_f(f_time_dep), "f"), int(f_time_dep),
                                          _ptr(u0, self.nx, "u0"), _ptr(x, self.n_st, "x"), int(x0_given),
                                          C.byref(info)),
                   allow=(-4,) if allow_not_converged else ())
        return x, Info.from_c(info)

    def solve_rhs(self, rhs, x, x0_given=False, allow_not_converged=False):
        """Solve A x = rhs for a given all-at-once right-hand side (n_st values)."""
        info = _lib.aao_info()
        _lib.check(self._lib.aao_rk_solve_rhs(self.h, _ptr(rhs, self.n_st, "rhs"), _ptr(x, self.n_st, "x"),
                                              int(x0_given), C.byref(info)),
                   allow=(-4,) if allow_not_converged else ())
        return x, Info.from_c(info)

    def adjoint_solve(self, dJdx, lam, x_fwd=None, grad_f=None, grad_kappa=None, allow_not_converged=False):
        """Solve A^T lam = dJdx (n_st) with P_tilde^T; optionally the gradients with respect to f (n_x) and,
        given the forward solution x_fwd, to the nodal kappa (prod(n + 2) values)."""
        info = _lib.aao_info()
        _lib.check(self._lib.aao_rk_adjoint_solve(self.h, _ptr(dJdx, self.n_st, "dJdx"), _ptr(lam, self.n_st, "lam"),
                                                  _ptr(x_fwd, self.n_st, "x_fwd"), _ptr(grad_f, self.nx, "grad_f"),
                                                  _ptr(grad_kappa, self.n_nodes, "grad_kappa"), C.byref(info)),
                   allow=(-4,) if allow_not_converged else ())
        return lam, Info.from_c(info)

    def grad_kappa(self, lam, x_fwd, out, accumulate=False):
        """out (+)= dJ/dkappa at the nodes from the adjoint lam and the forward solution x_fwd (n_st each)."""
        _lib.check(self._lib.aao_rk_grad_kappa(self.h, _ptr(lam, self.n_st, "lam"), _ptr(x_fwd, self.n_st, "x_fwd"),
                                               _ptr(out, self.n_nodes, "out"), int(accumulate)))
        return out


def solve_batched(solvers, fs, u0s, xs):
    """One call for many independent problems (aao_rk_solve_batched)."""
    lib = _lib.lib()
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s.h for s in solvers])
    if not (len(fs) == len(u0s) == len(xs) == n):
        raise ValueError("one f, u0 and x per solver")
    F = (C.c_void_p * n)(*[_ptr(f, s.nx, "f") for f, s in zip(fs, solvers)])
    U = (C.c_void_p * n)(*[_ptr(u, s.nx, "u0") for u, s in zip(u0s, solvers)])
    X = (C.c_void_p * n)(*[_ptr(x, s.n_st, "x") for x, s in zip(xs, solvers)])
    infos = (_lib.aao_info * n)()
    _lib.check(lib.aao_rk_solve_batched(n, hs, F, U, X, infos))
    return [Info.from_c(i) for i in infos]
