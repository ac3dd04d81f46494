"""The all-at-once RK operator of Eq. (system_all_at_once_RK), its transpose, rhs.

Test infrastructure only (see the package header).  Parity: pinned by the
dense Kronecker assembly of the four blocks, by the closed-form eigenmode
solution and by sequential RK time stepping (tests).

Unknown ordering (Sec. 2): x = [v_0 .. v_nt ; V_0 .. V_{nt-1}], V_n =
[V_{n,1} .. V_{n,s}], every block n_x long.  Block definitions (Sec. 2):

  Phi    = block-bidiagonal, M on the diagonal, -M below it   ((nt+1) x (nt+1))
  Psi_1  = -[0 ; tau b^T (x) M on the block sub-diagonal]     ((nt+1) x nt)
  Psi_2  = [e (x) K on the block diagonal, last column 0]      (nt x (nt+1))
  Theta  = I_nt (x) Theta_hat,  Theta_hat = I_s (x) M + tau A_RK (x) K

so, row by row,
  (A x)_{v,0}   = M v_0
  (A x)_{v,n+1} = M (v_{n+1} - v_n - tau sum_i b_i V_{n,i})
  (A x)_{V,n,i} = M V_{n,i} + K (v_n + tau sum_j a_ij V_{n,j}).

Right-hand side for zero Dirichlet data: b = [M u0 ; 0 ...] and f_{n,i} = M f
(f constant in time) or M f(t_n + c_i tau) when a time-dependent f is given.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class AllAtOnce:
    def __init__(self, K, M, tau: float, nt: int, A, b, c):
        self.K = sp.csr_matrix(K)
        self.M = None if M is None else sp.csr_matrix(M)
        self.tau = float(tau)
        self.nt = int(nt)
        self.A = np.asarray(A, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.s = len(self.b)
        self.nx = self.K.shape[0]
        self.n_v = (self.nt + 1) * self.nx
        self.n_st = self.n_v + self.nt * self.s * self.nx

    # -- helpers -----------------------------------------------------------
    def Mmul(self, u):
        return u.copy() if self.M is None else self.M @ u

    def MTmul(self, u):
        return u.copy() if self.M is None else self.M.T @ u

    def split(self, x):
        v = x[: self.n_v].reshape(self.nt + 1, self.nx)
        V = x[self.n_v:].reshape(self.nt, self.s, self.nx)
        return v, V

    def join(self, v, V):
        return np.concatenate([v.reshape(-1), V.reshape(-1)])

    # -- operator ------------------------------------------------------------
    def matvec(self, x):
        v, V = self.split(np.asarray(x, dtype=np.float64))
        yv = np.empty_like(v)
        yV = np.empty_like(V)
        tau, A, b = self.tau, self.A, self.b
        yv[0] = self.Mmul(v[0])
        for n in range(self.nt):
            acc = v[n + 1] - v[n]
            for i in range(self.s):
                acc = acc - tau * b[i] * V[n, i]
            yv[n + 1] = self.Mmul(acc)
            for i in range(self.s):
                W = v[n].copy()
                for j in range(self.s):
                    W = W + tau * A[i, j] * V[n, j]
                yV[n, i] = self.Mmul(V[n, i]) + self.K @ W
        return self.join(yv, yV)

    def rmatvec(self, lam):
        """A^T lam, from the transposed blocks [[Phi^T, Psi_2^T], [Psi_1^T, Theta^T]]."""
        lv, lV = self.split(np.asarray(lam, dtype=np.float64))
        ov = np.empty_like(lv)
        oV = np.empty_like(lV)
        tau, A, b = self.tau, self.A, self.b
        KT = self.K.T
        for n in range(self.nt + 1):
            acc = self.MTmul(lv[n])
            if n < self.nt:
                acc = acc - self.MTmul(lv[n + 1])
                for i in range(self.s):
                    acc = acc + KT @ lV[n, i]
            ov[n] = acc
        for n in range(self.nt):
            for i in range(self.s):
                acc = self.MTmul(lV[n, i]) - tau * b[i] * self.MTmul(lv[n + 1])
                for j in range(self.s):
                    acc = acc + tau * A[j, i] * (KT @ lV[n, j])
                oV[n, i] = acc
        return self.join(ov, oV)

    def rhs(self, u0, f, f_time_dep: bool = False):
        """[M u0 ; 0 ... ; f_{0,1} .. f_{nt-1,s}] for zero Dirichlet data."""
        v = np.zeros((self.nt + 1, self.nx))
        V = np.zeros((self.nt, self.s, self.nx))
        v[0] = self.Mmul(np.asarray(u0, dtype=np.float64))
        f = np.asarray(f, dtype=np.float64)
        if f_time_dep:
            F = f.reshape(self.nt, self.s, self.nx)
            for n in range(self.nt):
                for i in range(self.s):
                    V[n, i] = self.Mmul(F[n, i])
        else:
            Mf = self.Mmul(f)
            V[:, :, :] = Mf
        return self.join(v, V)

    # -- dense Kronecker assembly (tiny problems only) -----------------------
    def dense(self):
        nt, s, nx, tau = self.nt, self.s, self.nx, self.tau
        M = np.eye(nx) if self.M is None else self.M.toarray()
        K = self.K.toarray()
        Phi = np.kron(np.eye(nt + 1), M) - np.kron(np.eye(nt + 1, k=-1), M)
        E1 = np.zeros((nt + 1, nt))
        for n in range(nt):
            E1[n + 1, n] = 1.0
        Psi1 = -np.kron(E1, tau * np.kron(self.b[None, :], M))
        E2 = np.zeros((nt, nt + 1))
        for n in range(nt):
            E2[n, n] = 1.0
        Psi2 = np.kron(E2, np.kron(np.ones((s, 1)), K))
        Theta_hat = np.kron(np.eye(s), M) + tau * np.kron(self.A, K)
        Theta = np.kron(np.eye(nt), Theta_hat)
        return np.block([[Phi, Psi1], [Psi2, Theta]])

    def theta_hat(self):
        """Sparse Theta_hat = I_s (x) M + tau A (x) K."""
        M = sp.identity(self.nx, format="csr") if self.M is None else self.M
        return (sp.kron(sp.identity(self.s), M) + self.tau * sp.kron(self.A, self.K)).tocsr()


def dof_count(n_x: int, nt: int, s: int) -> int:
    """Space-time unknowns n_x (1 + nt (s + 1)) of Eq. (system_all_at_once_RK)."""
    return n_x * (1 + nt * (s + 1))
