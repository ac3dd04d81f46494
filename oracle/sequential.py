"""Sequential RK time stepping with direct stage solves (Sec. 2).

Test infrastructure only (see the package header).

For n = 0..nt-1: solve Theta_hat V_n = f_n - (e (x) K) v_n directly
(Eq. discretized_system_stages), then M v_{n+1} = M v_n + tau sum_i b_i M V_{n,i}
(Eq. update_solution), i.e. v_{n+1} = v_n + tau sum_i b_i V_{n,i}.  Its result
is, by construction, the solution of the all-at-once system; the tests use it
as an independent pin of the all-at-once operator and solver.
sequential_adjoint_rk is the same for the transposed system (backward in time),
pinned to a dense transposed solve and used to pin the FGMRES adjoint solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def sequential_rk(op, u0, f, f_time_dep=False):
    """Returns the all-at-once vector [v ; V] produced by time stepping."""
    nt, s, nx, tau, b = op.nt, op.s, op.nx, op.tau, op.b
    lu = spla.splu(op.theta_hat().tocsc())
    v = np.zeros((nt + 1, nx))
    V = np.zeros((nt, s, nx))
    v[0] = np.asarray(u0, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    for n in range(nt):
        if f_time_dep:
            fn = np.concatenate([op.Mmul(f.reshape(nt, s, nx)[n, i]) for i in range(s)])
        else:
            fn = np.tile(op.Mmul(f), s)
        Kv = op.K @ v[n]
        V[n] = lu.solve(fn - np.tile(Kv, s)).reshape(s, nx)
        v[n + 1] = v[n] + tau * sum(b[i] * V[n, i] for i in range(s))
    return op.join(v, V)


def sequential_adjoint_rk(op, g):
    """lambda = A^{-T} g by backward time stepping with direct stage solves.

    The columns of the all-at-once operator (Sec. 2) give, for lambda = [mu ; Lambda]:
      v_nt:     M^T mu_nt = g_{v,nt};
      V_{n,i}:  M^T Lambda_{n,i} + tau sum_j a_ji K^T Lambda_{n,j} - tau b_i M^T mu_{n+1} = g_{V,n,i},
                i.e. Theta_hat^T Lambda_n = g_{V,n} + tau (b (x) M^T) mu_{n+1};
      v_n:      M^T mu_n - M^T mu_{n+1} + K^T sum_i Lambda_{n,i} = g_{v,n}   (n < nt),
    solved for n = nt-1 .. 0 (the discrete adjoint of sequential RK stepping)."""
    nt, s, nx, tau, b = op.nt, op.s, op.nx, op.tau, op.b
    gv, gV = op.split(np.asarray(g, dtype=np.float64))
    lu = spla.splu(op.theta_hat().T.tocsc())
    luM = None if op.M is None else spla.splu(op.M.T.tocsc())
    solveMT = (lambda r: r.copy()) if luM is None else luM.solve
    mu = np.zeros((nt + 1, nx))
    Lam = np.zeros((nt, s, nx))
    mu[nt] = solveMT(gv[nt])
    for n in range(nt - 1, -1, -1):
        Mmu = op.MTmul(mu[n + 1])
        Lam[n] = lu.solve(np.concatenate([gV[n, i] + tau * b[i] * Mmu for i in range(s)])).reshape(s, nx)
        KL = sum(op.K.T @ Lam[n, i] for i in range(s))
        mu[n] = solveMT(gv[n] + Mmu - KL)
    return op.join(mu, Lam)


def sequential_solve(op, rhs):
    """x = A^{-1} rhs for any right-hand side by forward substitution in time with direct solves.

    The rows of the all-at-once operator (Sec. 2) give, for rhs = [r_v ; r_V]:
      M v_0 = r_{v,0};
      Theta_hat V_n = r_{V,n} - (e (x) K) v_n;
      M v_{n+1} = M v_n + tau sum_i b_i M V_{n,i} + r_{v,n+1}."""
    nt, s, nx, tau, b = op.nt, op.s, op.nx, op.tau, op.b
    rv, rV = op.split(np.asarray(rhs, dtype=np.float64))
    lu = spla.splu(op.theta_hat().tocsc())
    luM = None if op.M is None else spla.splu(op.M.tocsc())
    solveM = (lambda r: r.copy()) if luM is None else luM.solve
    v = np.zeros((nt + 1, nx))
    V = np.zeros((nt, s, nx))
    v[0] = solveM(rv[0])
    for n in range(nt):
        Kv = op.K @ v[n]
        V[n] = lu.solve(np.concatenate([rV[n, i] - Kv for i in range(s)])).reshape(s, nx)
        v[n + 1] = v[n] + tau * sum(b[i] * V[n, i] for i in range(s)) + solveM(rv[n + 1])
    return op.join(v, V)
