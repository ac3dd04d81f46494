"""Storage-precision emulation of P_tilde (Sec. 4, approaches A2, A4, A5; Sec. 5.1's rounding).

Test infrastructure only (see the package header).

The paper studies P_tilde applied in lower precision while the outer FGMRES stays in
FP64 (Sec. 4), and simulates the lower precision in its sequential runs by rounding
what is stored (Sec. 5.1).  This module restates that rounding for the storage
formats this implementation offers, so that a P_tilde kept in FP32, BF16 or FP16 can
be compared value by value with a run of the same definition, instead of only with
the FP64 result.  The steps are those of oracle.multigrid and oracle.precond (the
V-cycle, Rana's stage sweep, inner GMRES, the forward substitution of Eq. AppSchur);
only the precision of what they store and compute changes.

Reading (the paper fixes the idea, not the format details):

* fp32 storage: a stored value is float32(x), round to nearest, ties to even;
* bf16 / fp16 storage: a vector is a set of grid rows (n0 consecutive values along x
  of one stage of one time block); each row keeps one power-of-two scale
  s_row = 2^(e - 14) with 2^(e - 1) <= max|row| < 2^e (the maximum taken in
  float32), a value x is stored as RNE_p(x * 2^(14 - e)) and read back as
  stored * s_row; a zero row has scale 1;
* a Galerkin coarse stencil (one coefficient per point and neighbour offset) keeps one
  scale per offset, from the FP64 maximum over the level: stored = RNE_p(float32(a / s_q));
* every operation on stored values is a float32 operation (float64 for FP64 storage,
  where nothing is rounded);
* which intermediate vectors are stored and which stay in the arithmetic type between
  two steps is a property of the implementation under test (its memory plan), passed
  in as a `Plan` (see `StoredMG`).

Pins (tests): the BF16 and FP16 roundings against a brute-force search of each format's
values with ties to even; a row's scale is an exact power of two and its stored maximum
lies in [2^13, 2^14]; a stored value is within half a unit in the last place of the
format (times the row scale); with FP64 storage every emulated piece equals the plain
oracle (V-cycles, P_int, inner GMRES, P_tilde) to rounding level; FP32 and 16-bit
emulations stay within the error their unit roundoff allows of the FP64 oracle.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from .multigrid import Hierarchy
from .precond import Preconditioner, givens

FORMATS = ("fp64", "fp32", "bf16", "fp16")


# ---------------------------------------------------------------------------- roundings
def round_bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32)


def round_fp16(x):
    """float32 -> nearest IEEE half (ties to even), returned as float32 values."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def rne(x32, fmt):
    if fmt == "bf16":
        return round_bf16(x32)
    if fmt == "fp16":
        return round_fp16(x32)
    if fmt == "fp32":
        return np.asarray(x32, dtype=np.float32)
    raise ValueError(fmt)


def arith(fmt):
    """Arithmetic type of a storage format: float64 for fp64, float32 otherwise."""
    return np.float64 if fmt == "fp64" else np.float32


def row_scales(rows32):
    """Per-row power-of-two scale s and its inverse for 16-bit storage (rows: float32 2-D)."""
    m = np.abs(rows32).max(axis=1).astype(np.float32)
    ok = (m > 0) & (m <= np.float32(3.0e38))
    _, e = np.frexp(np.where(ok, m, np.float32(1)))
    e = e.astype(np.int64)
    one = np.float32(1)
    sc = np.where(ok, np.ldexp(one, e - 14), one).astype(np.float32)
    inv = np.where(ok, np.ldexp(one, 14 - e), one).astype(np.float32)
    return sc, inv


def store_rows(x, n0, fmt):
    """Values of x (computed in the arithmetic type) after storage in fmt, rows of n0."""
    if fmt == "fp64":
        return np.array(x, dtype=np.float64)
    x32 = np.asarray(x, dtype=np.float32)
    if fmt == "fp32":
        return x32.copy()
    rows = x32.reshape(-1, n0)
    sc, inv = row_scales(rows)
    stored = rne(rows * inv[:, None], fmt)
    return (stored * sc[:, None]).reshape(-1)


def stencil_scales(S64):
    """Per-component power-of-two scale of a stencil for 16-bit storage (from the FP64 maxima)."""
    sc = np.ones(S64.shape[0], dtype=np.float32)
    for q in range(S64.shape[0]):
        mm = float(np.abs(S64[q]).max())
        if mm > 0.0:
            _, e = np.frexp(mm)
            sc[q] = np.float32(np.ldexp(1.0, int(e) - 14))
    return sc


def store_stencil(S64, fmt):
    """A 3^d-point stencil (components x points, FP64) after storage in fmt."""
    S64 = np.asarray(S64, dtype=np.float64)
    if fmt == "fp64":
        return S64.copy()
    if fmt == "fp32":
        return S64.astype(np.float32)
    out = np.empty(S64.shape, dtype=np.float32)
    sc = stencil_scales(S64)
    for q in range(S64.shape[0]):
        out[q] = rne((S64[q] / np.float64(sc[q])).astype(np.float32), fmt) * sc[q]
    return out


# ---------------------------------------------------------------------------- stencils
def _offsets(d):
    offs = []
    for dz in ((-1, 0, 1) if d == 3 else (0,)):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offs.append((dx, dy, dz))
    return offs


def stencil_of(A, ns):
    """Components S[q, p] = A[p, p + offset_q] of a 3^d-point operator on grid ns (x fastest),
    q = (dx+1) + 3 (dy+1) [+ 9 (dz+1)]; zero where the neighbour is outside the grid."""
    ns = tuple(ns) + (1,) * (3 - len(ns))
    d = 3 if ns[2] > 1 or len(ns) == 3 and ns[2] > 1 else 2
    n0, n1, n2 = ns
    nx = n0 * n1 * n2
    A = sp.csr_matrix(A)
    i = np.arange(nx) % n0
    j = (np.arange(nx) // n0) % n1
    k = np.arange(nx) // (n0 * n1)
    offs = _offsets(3 if n2 > 1 else 2)
    S = np.zeros((len(offs), nx))
    for q, (dx, dy, dz) in enumerate(offs):
        ok = (i + dx >= 0) & (i + dx < n0) & (j + dy >= 0) & (j + dy < n1) & (k + dz >= 0) & (k + dz < n2)
        p = np.nonzero(ok)[0]
        S[q, p] = np.asarray(A[p, p + dx + n0 * (dy + n1 * dz)]).ravel()
    return S


def matrix_of(S, ns):
    """Sparse operator from stencil components (inverse of stencil_of)."""
    ns = tuple(ns) + (1,) * (3 - len(ns))
    n0, n1, n2 = ns
    nx = n0 * n1 * n2
    i = np.arange(nx) % n0
    j = (np.arange(nx) // n0) % n1
    k = np.arange(nx) // (n0 * n1)
    rows, cols, vals = [], [], []
    for q, (dx, dy, dz) in enumerate(_offsets(3 if n2 > 1 else 2)):
        ok = (i + dx >= 0) & (i + dx < n0) & (j + dy >= 0) & (j + dy < n1) & (k + dz >= 0) & (k + dz < n2)
        p = np.nonzero(ok)[0]
        rows.append(p)
        cols.append(p + dx + n0 * (dy + n1 * dz))
        vals.append(S[q, p])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx, nx), dtype=S.dtype)


# ---------------------------------------------------------------------------- multigrid
@dataclass
class Plan:
    """Memory plan of one multigrid solve: which vectors are stored between steps.

    onchip_from: levels l >= onchip_from run as one on-chip V-cycle (nothing stored inside it;
                 its b and x are read from and written to storage);
    fuse[l]:     above onchip_from, level l fuses two pre-smoothing sweeps, the residual with
                 the restriction, and the interpolation with the first post-smoothing sweep
                 (the intermediate results stay in the arithmetic type);
    keep_x:      all cycles of a solve on chip (x is stored once, after the last cycle).
    """
    onchip_from: int = 0
    fuse: List[bool] = field(default_factory=list)
    keep_x: bool = False


class StoredMG:
    """`cycles` V-cycles of oracle.multigrid.Hierarchy with storage in fmt (see module header).

    fine_stored: the finest level is a stored stencil too (Q1); otherwise its operator is the
    matrix-free one, evaluated in the arithmetic type."""

    def __init__(self, hier: Hierarchy, fmt: str, fine_stored: bool = False):
        self.h = hier
        self.fmt = fmt
        self.dt = arith(fmt)
        self.sizes = hier.sizes
        self.n0 = [s[0] for s in hier.sizes]
        L = hier.nlevels
        self.A, self.D = [], []
        for l in range(L):
            if l == 0 and not fine_stored:
                Al = hier.A[0].astype(self.dt)
            elif l < L - 1:
                Al = matrix_of(store_stencil(stencil_of(hier.A[l], self.sizes[l]), fmt), self.sizes[l])
            else:
                Al = None          # the coarsest level is solved through its dense inverse
            self.A.append(Al)
            self.D.append(None if Al is None else Al.diagonal().astype(self.dt))
        self.P = [P.astype(self.dt) for P in hier.P]
        self.Dinv = np.linalg.inv(hier.A[-1].toarray()).astype(self.dt)
        self.om = self.dt(hier.omega)

    def st(self, l, v):
        return store_rows(v, self.n0[l], self.fmt).astype(self.dt, copy=False)

    # pieces in the arithmetic type (x None: zero)
    def sweep(self, l, x, b):
        if x is None:
            return (self.om * b) / self.D[l]
        return x + (self.om * (b - self.A[l] @ x)) / self.D[l]

    def resid(self, l, x, b):
        return b.copy() if x is None else b - self.A[l] @ x

    def prolong(self, l, x, xc):
        return self.P[l] @ xc if x is None else x + self.P[l] @ xc

    def onchip(self, l, x, b):
        """One V-cycle of levels l.. with every vector in the arithmetic type."""
        L = self.h.nlevels
        if l == L - 1:
            return self.Dinv @ b
        for _ in range(self.h.nu1):
            x = self.sweep(l, x, b)
        bc = self.P[l].T @ self.resid(l, x, b)
        xc = self.onchip(l + 1, None, bc)
        x = self.prolong(l, x, xc)
        for _ in range(self.h.nu2):
            x = self.sweep(l, x, b)
        return x

    def stored(self, l, x, b, plan: Plan):
        """One V-cycle of levels l.. whose inputs and outputs are stored vectors."""
        if l >= min(plan.onchip_from, self.h.nlevels - 1):      # the coarsest level is always on chip
            return self.st(l, self.onchip(l, x, b))
        nu1, nu2 = self.h.nu1, self.h.nu2
        fuse = plan.fuse[l] if l < len(plan.fuse) else False
        q = 0
        if fuse and nu1 >= 2:
            x = self.st(l, self.sweep(l, self.sweep(l, x, b), b))
            q = 2
        for _ in range(q, nu1):
            x = self.st(l, self.sweep(l, x, b))
        if fuse or x is None:
            bc = self.st(l + 1, self.P[l].T @ self.resid(l, x, b))
        else:
            r = self.st(l, self.resid(l, x, b))
            bc = self.st(l + 1, self.P[l].T @ r)
        xc = self.stored(l + 1, None, bc, plan)
        if fuse and nu2 >= 1:
            x = self.st(l, self.sweep(l, self.prolong(l, x, xc), b))
            q = 1
        else:
            x = self.st(l, self.prolong(l, x, xc))
            q = 0
        for _ in range(q, nu2):
            x = self.st(l, self.sweep(l, x, b))
        return x

    def solve(self, b, cycles: int, plan: Plan):
        """x after `cycles` V-cycles from zero; b holds stored values, x is returned stored."""
        b = np.asarray(b, dtype=self.dt)
        x = None
        if plan.keep_x:
            for _ in range(cycles):
                x = self.onchip(0, x, b)
            return self.st(0, x)
        for _ in range(cycles):
            x = self.stored(0, x, b, plan)
        return x


# ---------------------------------------------------------------------------- P_tilde
class StoredPreconditioner:
    """P_tilde of oracle.precond.Preconditioner (FD, M = I) with Theta_tilde's GMRES basis and the
    S_tilde recurrence in fmt_P and Rana's sweep, the V-cycles and coarse stencils in fmt_I.

    plan_batch is the multigrid memory plan of the batched Theta_tilde phase (all time blocks at
    once), plan_single that of single-block solves (the S_tilde sweep and the component calls)."""

    def __init__(self, P: Preconditioner, fmt_P: str, fmt_I: str, plan_batch: Plan, plan_single: Plan):
        if P.op.M is not None or P.exact:
            raise ValueError("the storage emulation covers the FD preconditioner with multigrid")
        if (fmt_P == "fp64") != (fmt_I == "fp64"):
            raise ValueError("FP64 storage is all or nothing")
        self.P = P
        self.op = P.op
        self.fP, self.fI = fmt_P, fmt_I
        self.dt = arith(fmt_I)
        self.n0 = P.ns[0]
        self.mg = [StoredMG(h, fmt_I) for h in P.mg]
        self.K = P.op.K.astype(self.dt)
        self.plan_batch, self.plan_single = plan_batch, plan_single
        self.inner_its = 0

    def stP(self, v):
        return store_rows(v, self.n0, self.fP).astype(self.dt, copy=False)

    def stI(self, v):
        return store_rows(v, self.n0, self.fI).astype(self.dt, copy=False)

    def shifted_solve(self, i, b_stored, plan):
        return self.mg[i].solve(b_stored, self.P.mg_cycles, plan)

    def pint(self, V, plan, transpose=False):
        """Z = P_int^{-1} V (stage rows of stored values), forward (or backward) stage sweep."""
        s, dt, tau = self.op.s, self.dt, self.dt(self.op.tau)
        LD = self.P.LD
        V = V.reshape(s, -1)
        Z = np.zeros(V.shape, dtype=dt)
        order = range(s - 1, -1, -1) if transpose else range(s)
        for i in order:
            acc = V[i].astype(dt)
            for j in range(s):
                cf = LD[j, i] if transpose else LD[i, j]
                if (j > i if transpose else j < i) and cf != 0.0:
                    acc = acc - (tau * dt(cf)) * (self.K @ Z[j])
            Z[i] = self.shifted_solve(i, self.stI(acc), plan)
        return Z.reshape(-1)

    def theta(self, z, transpose=False):
        """w = Theta_hat z (or Theta_hat^T z) in the arithmetic type, z of stored values."""
        s, dt, tau = self.op.s, self.dt, self.dt(self.op.tau)
        A = self.op.A.T if transpose else self.op.A
        Z = z.reshape(s, -1)
        KZ = [self.K @ Z[j] for j in range(s)]
        out = np.empty(Z.shape, dtype=dt)
        for i in range(s):
            acc = Z[i].copy()
            for j in range(s):
                acc = acc + (tau * dt(A[i, j])) * KZ[j]
            out[i] = acc
        return out.reshape(-1)

    def inner(self, r, plan, transpose=False):
        """Inner GMRES(k) on Theta_hat for one block (oracle.precond.gmres_fixed with stored bases).
        Returns (y, Z, its): the least-squares coefficients and the stored P_int directions."""
        dt = self.dt
        kin, tol = self.P.inner_maxit, self.P.inner_tol
        beta = float(np.sqrt(np.dot(np.asarray(r, np.float64), np.asarray(r, np.float64))))
        if not beta > 0.0:
            return np.zeros(0), [], 0
        inv = dt(1) / dt(beta)
        V = [self.stP(np.asarray(r, dtype=dt) * inv)]
        Z = []
        H = np.zeros((kin + 1, kin))
        cs, sn, g = np.zeros(kin), np.zeros(kin), np.zeros(kin + 1)
        g[0] = beta
        its = 0
        for k in range(kin):
            Z.append(self.pint(V[k], plan, transpose))
            w = self.theta(Z[k], transpose)
            H[0, k] = float(np.dot(V[0].astype(np.float64), w.astype(np.float64)))
            for i in range(1, k + 2):
                w = w - dt(H[i - 1, k]) * V[i - 1]
                if i <= k:
                    H[i, k] = float(np.dot(V[i].astype(np.float64), w.astype(np.float64)))
                else:
                    H[i, k] = float(np.sqrt(np.dot(w.astype(np.float64), w.astype(np.float64))))
            hk1 = H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            cs[k], sn[k], H[k, k] = givens(H[k, k], hk1)
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its = k + 1
            if abs(g[k + 1]) <= tol * beta or hk1 == 0.0 or k == kin - 1:
                break
            V.append(self.stP(w * (dt(1) / dt(hk1))))
        y = np.zeros(its)
        for i in range(its - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:its] @ y[i + 1:its]) / H[i, i]
        self.inner_its += its
        return y, Z, its

    def combine(self, y, Z, n):
        acc = np.zeros(n, dtype=self.dt)
        for k in range(len(y)):
            acc = acc + self.dt(y[k]) * Z[k]
        return acc.astype(np.float64)

    def inner_solve(self, r, plan, transpose=False):
        """z = Theta_tilde^{-1} r for one block (FP64 in and out)."""
        y, Z, _ = self.inner(r, plan, transpose)
        return self.combine(y, Z, len(r))

    def apply(self, r):
        """z = P_tilde^{-1} r (FP64 in and out): batched Theta_tilde phase, Schur right-hand side
        w, then the forward substitution of Eq. (AppSchur) one time step at a time."""
        op, dt = self.op, self.dt
        nt, s, nx, tau, b = op.nt, op.s, op.nx, op.tau, op.b
        rv, rV = op.split(np.asarray(r, dtype=np.float64))
        zV = np.stack([self.inner_solve(rV[n].reshape(-1), self.plan_batch) for n in range(nt)])
        zV = zV.reshape(nt, s, nx)
        w = np.empty((nt + 1, nx), dtype=dt)
        w[0] = rv[0].astype(dt)
        for n in range(nt):
            acc = np.zeros(nx, dtype=dt)
            for q in range(s):
                acc = acc + dt(b[q]) * zV[n, q].astype(dt)
            w[n + 1] = rv[n + 1].astype(dt) + dt(tau) * acc
        zv = np.empty((nt + 1, nx))
        zv[0] = w[0].astype(np.float64)
        for n in range(nt):
            t = np.tile((op.K @ zv[n]).astype(dt), s)
            y, Z, _ = self.inner(t, self.plan_single)
            acc = w[n + 1] + zv[n].astype(dt)
            for k in range(len(y)):
                Zk = Z[k].reshape(s, nx)
                for i in range(s):
                    acc = acc - dt(tau * b[i] * y[k]) * Zk[i]
            zv[n + 1] = acc.astype(np.float64)
        return op.join(zv, zV)

    def apply_T(self, r):
        """z = P_tilde^{-T} r (FP64 in and out): the backward substitution of S_tilde^T one time step
        at a time, then the batched Theta_tilde^{-T} phase on r_V - Psi_1^T z_v."""
        op, dt = self.op, self.dt
        nt, s, nx, tau, b = op.nt, op.s, op.nx, op.tau, op.b
        rv, rV = op.split(np.asarray(r, dtype=np.float64))
        u = np.empty((nt + 1, nx))
        u[nt] = rv[nt]
        for n in range(nt - 1, -1, -1):
            un1 = u[n + 1].astype(dt)
            t = np.concatenate([dt(b[q]) * un1 for q in range(s)])
            y, Z, _ = self.inner(t, self.plan_single, transpose=True)
            qv = self.combine(y, Z, s * nx).astype(dt).reshape(s, nx)
            acc = np.zeros(nx, dtype=dt)
            for i in range(s):
                acc = acc + self.K @ qv[i]
            u[n] = (rv[n].astype(dt) + un1 - dt(tau) * acc).astype(np.float64)
        zV = np.empty((nt, s, nx))
        for n in range(nt):
            t = np.concatenate([rV[n, q].astype(dt) + (dt(tau) * dt(b[q])) * u[n + 1].astype(dt)
                                for q in range(s)])
            zV[n] = self.inner_solve(t, self.plan_batch, transpose=True).reshape(s, nx)
        return op.join(u, zV)
