"""The block-triangular preconditioner P_tilde of Eq. (AppPrec) and its pieces.

Test infrastructure only (see the package header).

Sec. 3 and Fig. 1 (Sec. 5):
  P_tilde = [[S_tilde, Psi_1], [0, Theta_tilde]],
  Theta_tilde^{-1}: per time step, a few GMRES iterations on Theta_hat,
      right-preconditioned by Rana's stage preconditioner P_int;
  S_tilde = blkdiag(M) L_S, L_S unit block-lower-bidiagonal with sub-blocks
      -I + X_tilde, X_tilde = tau (b^T (x) I) Theta_tilde^{-1} (e (x) K)
      (Eq. AppSchur); applying it is a forward substitution in time;
  M^{-1} is 20 Chebyshev semi-iteration steps with Jacobi splitting (Q1) or
      the identity (FD);
  (M + cK)^{-1} is 3 multigrid V-cycles.

Reading of Rana's preconditioner (not defined in the paper): the block-LDU
preconditioner A_RK = L D U, P_int = I (x) M + tau (L D) (x) K, block lower
triangular with diagonal blocks M + tau d_i K; applying it is a forward
sweep over the stages.

Solving P_tilde z = r (block back-substitution):
  z_V = Theta_tilde^{-1} r_V;
  g_0 = r_{v,0}, g_{n+1} = r_{v,n+1} + tau sum_i b_i M z_{V,n,i}   (r_v - Psi_1 z_V);
  w = M^{-1} g;  z_{v,0} = w_0;
  z_{v,n+1} = w_{n+1} + z_{v,n} - tau sum_i b_i [Theta_tilde^{-1} (e (x) K z_{v,n})]_i.

Transposed preconditioner (adjoint solves): P_tilde^T = [[S^T, 0], [Psi_1^T, Theta^T]];
S^T = L_S^T blkdiag(M): backward substitution u_nt = g_nt,
u_n = g_n + u_{n+1} - tau (e^T (x) K) Theta_tilde^{-T} (b (x) u_{n+1}), z_v = M^{-1} u;
then z_V = Theta_tilde^{-T} (r_V - Psi_1^T z_v), (Psi_1^T z_v)_{n,i} = -tau b_i M z_{v,n+1}.
Theta_tilde^{-T} is inner GMRES on Theta_hat^T right-preconditioned by P_int^T
(a backward stage sweep).

With schur="mgrit" the time recurrences of S_tilde and S_tilde^T are solved
approximately by two-level MGRIT (module mgrit), as in the paper's parallel
implementation (Sec. 5); the fine step is the substitution step above, the
coarse step the same with step size m tau.

Parity: pinned by the exact-inverse limit (Theta_tilde = Theta_hat, exact
M^{-1}: FGMRES converges in <= 2 iterations, Sec. 3) and, for P_int, by the
s = 1 limit and a dense block-triangular solve (tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mgrit
from .aao import AllAtOnce
from .multigrid import Hierarchy
from .tableau import ldu
from .operators import q1_jacobi_interval


def givens(a: float, b: float):
    den = float(np.hypot(a, b))
    if den == 0.0:
        return 1.0, 0.0, 0.0
    return a / den, b / den, den


def gmres_fixed(apply_A, apply_P, r, maxit: int, tol: float):
    """GMRES(maxit) from x0 = 0, right-preconditioned, MGS, Z stored.

    Stops after `maxit` iterations or when the least-squares residual
    |g_{k+1}| <= tol * ||r||.  Returns (z, iterations).
    """
    beta = float(np.linalg.norm(r))
    if beta == 0.0:
        return np.zeros_like(r), 0
    V = [r / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    its = 0
    for k in range(maxit):
        Z.append(apply_P(V[k]))
        w = apply_A(Z[k])
        for i in range(k + 1):
            H[i, k] = float(V[i] @ w)
            w = w - H[i, k] * V[i]
        H[k + 1, k] = float(np.linalg.norm(w))
        for i in range(k):
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        hkk, hk1 = H[k, k], H[k + 1, k]
        cs[k], sn[k], H[k, k] = givens(hkk, hk1)
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        its = k + 1
        if abs(g[k + 1]) <= tol * beta or hk1 == 0.0 or k == maxit - 1:
            break
        V.append(w / hk1)
    y = np.zeros(its)
    for i in range(its - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:its] @ y[i + 1:its]) / H[i, i]
    z = np.zeros_like(r)
    for i in range(its):
        z = z + y[i] * Z[i]
    return z, its


class Preconditioner:
    """P_tilde for an AllAtOnce operator on grid `ns`.

    exact=True replaces every inner approximation by a direct solve
    (Theta_tilde = Theta_hat, exact M^{-1}, exact shifted solves).
    """

    def __init__(self, op, ns, inner_maxit=3, inner_tol=1e-3, mg_cycles=3, nu1=2, nu2=2,
                 omega=2.0 / 3.0, cheb_steps=20, exact=False, schur="sequential", mgrit_m=8,
                 mgrit_iters=1, mgrit_relax="FCF", mgrit_levels=2):
        self.op = op
        self.ns = tuple(ns)
        self.s, self.nt, self.nx = op.s, op.nt, op.nx
        self.inner_maxit, self.inner_tol = int(inner_maxit), float(inner_tol)
        self.mg_cycles = int(mg_cycles)
        self.cheb_steps = int(cheb_steps)
        self.exact = bool(exact)
        L, D, U = ldu(op.A)
        self.L, self.D, self.U = L, D, U
        self.LD = L @ np.diag(D)
        M = sp.identity(self.nx, format="csr") if op.M is None else op.M
        self.Msp = M
        self.shift = op.tau * D
        self.shifted = [(M + c * op.K).tocsr() for c in self.shift]
        if exact:
            self.lu_shift = [spla.splu(A.tocsc()) for A in self.shifted]
            self.lu_theta = spla.splu(op.theta_hat().tocsc())
            self.lu_M = None if op.M is None else spla.splu(op.M.tocsc())
        else:
            self.mg = [Hierarchy(A, self.ns, omega, nu1, nu2) for A in self.shifted]
        self.inner_its = 0
        # S_tilde's time recurrence: forward substitution (Eq. AppSchur) or, as in the paper's
        # parallel implementation (Sec. 5), MGRIT with the same step on the fine level and the
        # step of size m tau (nt / m steps) on the coarse level
        if schur not in ("sequential", "mgrit"):
            raise ValueError("schur is 'sequential' or 'mgrit'")
        self.schur = schur
        self.mgrit_m, self.mgrit_iters, self.mgrit_relax = int(mgrit_m), int(mgrit_iters), mgrit_relax
        self.mgrit_levels = int(mgrit_levels)
        self.coarse = None
        self.coarser = []          # levels 1 .. mgrit_levels-1: steps of size m^k tau
        if schur == "mgrit":
            if self.mgrit_levels < 2 or self.mgrit_m < 1 or self.mgrit_m > self.nt:
                raise ValueError("the MGRIT coarsening factor m must lie in 1 .. nt")
            # two levels take any m (a shorter final interval when m does not divide nt); the
            # multilevel cycle needs m^(levels-1) to divide nt
            if self.mgrit_levels > 2 and self.nt % self.mgrit_m ** (self.mgrit_levels - 1) != 0:
                raise ValueError("the MGRIT coarsening factor m (to the power levels-1) must divide nt")
            for k in range(1, self.mgrit_levels):
                mk = self.mgrit_m ** k
                op_k = AllAtOnce(op.K, op.M, mk * op.tau, self.nt // mk, op.A, op.b, op.c)
                self.coarser.append(Preconditioner(op_k, ns, inner_maxit, inner_tol, mg_cycles, nu1, nu2, omega,
                                                   cheb_steps, exact))
            self.coarse = self.coarser[0]

    # -- spatial pieces -------------------------------------------------------
    def shifted_solve(self, i, r):
        if self.exact:
            return self.lu_shift[i].solve(r)
        return self.mg[i].solve(r, self.mg_cycles)

    def mass_inverse(self, g):
        """M^{-1} g: identity (FD), exact, or Chebyshev semi-iteration (Q1)."""
        if self.op.M is None:
            return g.copy()
        if self.exact:
            return self.lu_M.solve(g)
        interval = getattr(self.op, "mass_interval", None) or q1_jacobi_interval(len(self.ns))
        return chebyshev_jacobi(self.op.M, g, self.cheb_steps, *interval)

    # -- stage pieces ---------------------------------------------------------
    def theta_apply(self, z):
        """Theta_hat z: w_i = M z_i + tau sum_j a_ij K z_j."""
        Z = z.reshape(self.s, self.nx)
        KZ = [self.op.K @ Z[j] for j in range(self.s)]
        out = np.empty_like(Z)
        for i in range(self.s):
            acc = self.op.Mmul(Z[i])
            for j in range(self.s):
                acc = acc + self.op.tau * self.op.A[i, j] * KZ[j]
            out[i] = acc
        return out.reshape(-1)

    def theta_apply_T(self, z):
        Z = z.reshape(self.s, self.nx)
        KZ = [self.op.K.T @ Z[j] for j in range(self.s)]
        out = np.empty_like(Z)
        for i in range(self.s):
            acc = self.op.MTmul(Z[i])
            for j in range(self.s):
                acc = acc + self.op.tau * self.op.A[j, i] * KZ[j]
            out[i] = acc
        return out.reshape(-1)

    def pint_apply(self, r):
        """y = P_int^{-1} r by the forward stage sweep."""
        R = r.reshape(self.s, self.nx)
        Y = np.zeros_like(R)
        for i in range(self.s):
            rhs = R[i].copy()
            for j in range(i):
                rhs = rhs - self.op.tau * self.LD[i, j] * (self.op.K @ Y[j])
            Y[i] = self.shifted_solve(i, rhs)
        return Y.reshape(-1)

    def pint_apply_T(self, r):
        """y = P_int^{-T} r by the backward stage sweep."""
        R = r.reshape(self.s, self.nx)
        Y = np.zeros_like(R)
        for i in range(self.s - 1, -1, -1):
            rhs = R[i].copy()
            for j in range(i + 1, self.s):
                rhs = rhs - self.op.tau * self.LD[j, i] * (self.op.K.T @ Y[j])
            Y[i] = self.shifted_solve(i, rhs)
        return Y.reshape(-1)

    def inner_solve(self, r, transpose=False):
        """Theta_tilde^{-1} r (or Theta_tilde^{-T} r) for one time step."""
        if self.exact:
            return (self.lu_theta.solve(r, trans="T" if transpose else "N"))
        if transpose:
            z, its = gmres_fixed(self.theta_apply_T, self.pint_apply_T, r,
                                 self.inner_maxit, self.inner_tol)
        else:
            z, its = gmres_fixed(self.theta_apply, self.pint_apply, r,
                                 self.inner_maxit, self.inner_tol)
        self.inner_its += its
        return z

    def theta_tilde(self, rV):
        """Block-diagonal Theta_tilde^{-1} over all time steps; rV shape (nt, s*nx)."""
        return np.stack([self.inner_solve(rV[n]) for n in range(self.nt)])

    # -- full preconditioner --------------------------------------------------
    def apply(self, r):
        """z = P_tilde^{-1} r."""
        op = self.op
        rv, rV = op.split(np.asarray(r, dtype=np.float64))
        nt, s, nx, tau, b = self.nt, self.s, self.nx, op.tau, op.b
        zV = self.theta_tilde(rV.reshape(nt, s * nx)).reshape(nt, s, nx)
        g = np.empty_like(rv)
        g[0] = rv[0]
        for n in range(nt):
            acc = np.zeros(nx)
            for i in range(s):
                acc = acc + b[i] * zV[n, i]
            g[n + 1] = rv[n + 1] + tau * op.Mmul(acc)
        w = np.stack([self.mass_inverse(g[n]) for n in range(nt + 1)])
        if self.schur == "mgrit":
            if self.mgrit_levels == 2:
                zv = mgrit.two_level(self.schur_step, self.coarse.schur_step, w, self.mgrit_m,
                                     self.mgrit_iters, self.mgrit_relax)
            else:
                zv = mgrit.multilevel([self.schur_step] + [c.schur_step for c in self.coarser], w,
                                      self.mgrit_m, self.mgrit_iters, self.mgrit_relax)
            return op.join(zv, zV)
        zv = np.empty_like(rv)
        zv[0] = w[0]
        for n in range(nt):
            t = np.tile(op.K @ zv[n], s)
            q = self.inner_solve(t).reshape(s, nx)
            acc = w[n + 1] + zv[n]
            for i in range(s):
                acc = acc - tau * b[i] * q[i]
            zv[n + 1] = acc
        return op.join(zv, zV)

    def schur_step(self, z):
        """One step of S_tilde's recurrence without its source: z - tau (b^T (x) I)
        Theta_tilde^{-1} (e (x) K z)."""
        q = self.inner_solve(np.tile(self.op.K @ z, self.s)).reshape(self.s, self.nx)
        acc = z.copy()
        for i in range(self.s):
            acc = acc - self.op.tau * self.op.b[i] * q[i]
        return acc

    def schur_step_T(self, u):
        """One step of S_tilde^T's backward recurrence without its source: u - tau (e^T (x) K^T)
        Theta_tilde^{-T} (b (x) u)."""
        q = self.inner_solve(np.concatenate([self.op.b[i] * u for i in range(self.s)]),
                             transpose=True).reshape(self.s, self.nx)
        acc = np.zeros(self.nx)
        for i in range(self.s):
            acc = acc + self.op.K.T @ q[i]
        return u - self.op.tau * acc

    def apply_T(self, r):
        """z = P_tilde^{-T} r."""
        op = self.op
        rv, rV = op.split(np.asarray(r, dtype=np.float64))
        nt, s, nx, tau, b = self.nt, self.s, self.nx, op.tau, op.b
        if self.schur == "mgrit":
            # the backward recurrence is a forward one in reversed time
            if self.mgrit_levels == 2:
                u = mgrit.two_level(self.schur_step_T, self.coarse.schur_step_T, rv[::-1], self.mgrit_m,
                                    self.mgrit_iters, self.mgrit_relax)[::-1]
            else:
                u = mgrit.multilevel([self.schur_step_T] + [c.schur_step_T for c in self.coarser], rv[::-1],
                                     self.mgrit_m, self.mgrit_iters, self.mgrit_relax)[::-1]
        else:
            u = np.empty_like(rv)
            u[nt] = rv[nt]
            for n in range(nt - 1, -1, -1):
                t = np.concatenate([b[i] * u[n + 1] for i in range(s)])
                q = self.inner_solve(t, transpose=True).reshape(s, nx)
                acc = np.zeros(nx)
                for i in range(s):
                    acc = acc + op.K.T @ q[i]
                u[n] = rv[n] + u[n + 1] - tau * acc
        zv = np.stack([self.mass_inverse_T(u[n]) for n in range(nt + 1)])
        zV = np.empty_like(rV)
        for n in range(nt):
            t = rV[n].copy()
            for i in range(s):
                t[i] = t[i] + tau * b[i] * op.MTmul(zv[n + 1])
            zV[n] = self.inner_solve(t.reshape(-1), transpose=True).reshape(s, nx)
        return op.join(zv, zV)

    def mass_inverse_T(self, g):
        # M is symmetric for both discretisations; Chebyshev with Jacobi is symmetric too
        return self.mass_inverse(g)


def chebyshev_jacobi(M, g, steps, lo, hi):
    """`steps` Chebyshev semi-iterations for M x = g, Jacobi splitting, x0 = 0.

    Chebyshev acceleration of the Jacobi-preconditioned iteration for an
    SPD M whose D^{-1}M spectrum lies in [lo, hi] (Golub--Varga; Saad,
    'Iterative Methods for Sparse Linear Systems', Alg. 12.1).
    """
    Dinv = 1.0 / M.diagonal()
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(g)
    r = g.copy()
    d = Dinv * r / theta
    for _ in range(steps):
        x = x + d
        r = r - M @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * r)
        rho = rho_new
    return x
