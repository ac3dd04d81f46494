"""Sequential RK time stepping with direct stage solves (Sec. 2).

Test infrastructure only (see the package header).

For n = 0..nt-1: solve Theta_hat V_n = f_n - (e (x) K) v_n directly
(Eq. discretized_system_stages), then M v_{n+1} = M v_n + tau sum_i b_i M V_{n,i}
(Eq. update_solution), i.e. v_{n+1} = v_n + tau sum_i b_i V_{n,i}.  Its result
is, by construction, the solution of the all-at-once system; the tests use it
as an independent pin of the all-at-once operator and solver.
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
