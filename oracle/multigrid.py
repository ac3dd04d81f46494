"""Geometric Galerkin multigrid V-cycles for the shifted operators M + cK.

Test infrastructure only (see the package header).

Sec. 5 approximates (M + cK)^{-1} by 3 cycles of the closed AMG code
HSL_MI20.  That code is not available, so the method here is a geometric
V-cycle with a fixed definition (shared with the GPU path as a definition,
not as code):

* per axis, fine interior indices 1..N; coarse points are the even fine
  indices, N_c = floor(N / 2); coarse j sits at fine 2j;
* 1D interpolation P: injection at coarse points; an odd fine point takes
  the average of its two neighbours, a Dirichlet boundary neighbour
  (index 0 or N+1) counting as 0; P = tensor product of the 1D P's;
* restriction R = P^T, coarse operator A_c = P^T A P (Galerkin);
* coarsen all axes together while the level has more than COARSEST_MAX = 256
  unknowns and every axis keeps N_c >= 2; the coarsest level is solved
  exactly (dense Cholesky);
* smoother: damped Jacobi x <- x + omega D^{-1} (b - A x), nu1 sweeps before
  and nu2 after the coarse correction;
* a solve runs `cycles` V-cycles from a zero initial guess, so it is a
  fixed linear operator.

Pins (tests): Galerkin coarse stencil of the constant-coefficient operator
against its tensor-product closed form; symmetry of the V-cycle operator for
nu1 = nu2; contraction factor on Poisson-type shifts; exact coarsest solve.
"""
from __future__ import annotations

from functools import reduce

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


COARSEST_MAX = 256   # a level with at most this many unknowns is solved exactly


def coarse_size(n: int) -> int:
    return n // 2


def interp_1d(n: int) -> sp.csr_matrix:
    """1D interpolation from N_c = N//2 coarse points to N fine points."""
    nc = coarse_size(n)
    rows, cols, vals = [], [], []
    for j in range(1, nc + 1):          # 1-based coarse index, fine index 2j
        f = 2 * j
        rows.append(f - 1); cols.append(j - 1); vals.append(1.0)
        for g in (f - 1, f + 1):
            if 1 <= g <= n:
                rows.append(g - 1); cols.append(j - 1); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))


def level_sizes(ns):
    """Per-level interior sizes, finest first."""
    sizes = [tuple(ns)]
    while int(np.prod(sizes[-1])) > COARSEST_MAX and all(coarse_size(n) >= 2 for n in sizes[-1]):
        sizes.append(tuple(coarse_size(n) for n in sizes[-1]))
    return sizes


class Hierarchy:
    def __init__(self, A0, ns, omega: float = 2.0 / 3.0, nu1: int = 2, nu2: int = 2):
        self.sizes = level_sizes(ns)
        self.omega, self.nu1, self.nu2 = float(omega), int(nu1), int(nu2)
        self.A = [sp.csr_matrix(A0)]
        self.P = []
        for l in range(1, len(self.sizes)):
            fine = self.sizes[l - 1]
            P = reduce(lambda X, Y: sp.kron(X, Y, format="csr"),
                       [interp_1d(n) for n in reversed(fine)])
            Ac = (P.T @ self.A[-1] @ P).tocsr()
            self.P.append(P.tocsr())
            self.A.append(Ac)
        self.D = [A.diagonal() for A in self.A]
        self.coarse_chol = sla.cho_factor(self.A[-1].toarray())

    @property
    def nlevels(self):
        return len(self.A)

    def smooth(self, l, x, b, sweeps):
        A, D, w = self.A[l], self.D[l], self.omega
        for _ in range(sweeps):
            x = x + w * (b - A @ x) / D
        return x

    def vcycle(self, l, x, b):
        if l == self.nlevels - 1:
            return sla.cho_solve(self.coarse_chol, b)
        x = self.smooth(l, x, b, self.nu1)
        r = b - self.A[l] @ x
        bc = self.P[l].T @ r
        xc = self.vcycle(l + 1, np.zeros(bc.shape[0]), bc)
        x = x + self.P[l] @ xc
        x = self.smooth(l, x, b, self.nu2)
        return x

    def solve(self, b, cycles: int = 3):
        x = np.zeros_like(b)
        for _ in range(cycles):
            x = self.vcycle(0, x, b)
        return x
