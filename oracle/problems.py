"""The paper's sequential test problem (Sec. 5.1) with Q1 or Q2 elements.

Test infrastructure only (see the package header).

Problem: the heat equation on [-1, 1]^2 up to t_f = 2 with exact solution
    v(x, t) = exp(t_f - t) cos(pi x_1 / 2) cos(pi x_2 / 2) + 1
(reading: the printed formula drops the second cosine; with both factors v = 1 on the boundary,
the data g = 1 the paper derives).  Writing v = 1 + w, w solves the heat equation with zero
Dirichlet data and source f = w_t - Delta w = (pi^2 / 2 - 1) w; w and v share the discretisation
error.  Coordinates are shifted to [0, 2]^2, X = x + 1, where cos(pi x / 2) = sin(pi X / 2).

Discretisation (Sec. 5): for refinement level l the element size is H = 2^(1-l) (2^l elements per
axis; interior nodes 2^l - 1 for Q1, 2^(l+1) - 1 for Q2, which reproduces every DoF cell of
Table 2); q_FE = 2 (Q1) or 3 (Q2), q_RK = 2s - 1 (Radau IIA), and n_t is the smallest integer with
tau = t_f / n_t <= H^(q_FE / q_RK).  Right-hand side (reading): the initial block is M times the
nodal interpolant of w(., 0); each stage block is the FE load vector of f at the stage time,
int f(., t_n + c_i tau) phi_j, integrated per element by Gauss--Legendre quadrature (`quad` points
per axis; the default 8 is exact to rounding for this smooth source).

Error (Sec. 5.1): v_error = max_n |v_{j,n} - v^sol_{j,n}| / |v^sol_{j,n}| with j the node of largest
absolute error at t_n, v^sol the nodal values of the exact solution.

Parity: pinned (tests) against the v_error values printed in Table 2 and by the convergence
orders in h; the discrete solution comes from sequential RK stepping with direct stage solves,
itself pinned to the all-at-once system.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .aao import AllAtOnce
from .operators import operators, q1_jacobi_interval, q2_jacobi_interval
from .tableau import tableau

T_FINAL = 2.0
LENGTH = 2.0


def level_nodes(disc: str, l: int) -> int:
    """Interior nodes per axis at refinement level l."""
    return 2 ** l - 1 if disc == "q1" else 2 ** (l + 1) - 1


def time_steps(disc: str, l: int, s: int, tf: float = T_FINAL) -> int:
    """Smallest n_t with tf / n_t <= H^(q_FE / q_RK), H = 2^(1-l), Radau IIA order 2s - 1."""
    q_fe = 2 if disc == "q1" else 3
    H = 2.0 ** (1 - l)
    return math.ceil(tf / H ** (q_fe / (2 * s - 1)) - 1e-9)


def _local_basis(disc: str, t: np.ndarray):
    """Values of the element's local basis functions at reference points t in [0, 1]."""
    if disc == "q1":
        return [1.0 - t, t]
    return [2.0 * (t - 0.5) * (t - 1.0), -4.0 * t * (t - 1.0), 2.0 * t * (t - 0.5)]


def load_1d(disc: str, n: int, func, length: float = LENGTH, quad: int = 8) -> np.ndarray:
    """int_0^length func(X) phi_j(X) dX for the interior nodal basis functions phi_j."""
    per = 1 if disc == "q1" else 2                   # node steps per element
    E = (n + 1) // per
    H = length / E
    gx, gw = np.polynomial.legendre.leggauss(quad)
    t = (gx + 1.0) / 2.0
    F = np.zeros(per * E + 1)
    for e in range(E):
        vals = func((e + t) * H) * gw * (H / 2.0)
        for k, phi in enumerate(_local_basis(disc, t)):
            F[per * e + k] += float(np.sum(vals * phi))
    return F[1:-1]


@dataclass
class ExactSolutionProblem:
    disc: str
    l: int
    s: int
    op: AllAtOnce
    n: int
    profile: np.ndarray        # sin(pi X / 2) sin(pi Y / 2) at the interior nodes (x fastest)
    load_profile: np.ndarray   # its load vector int sin sin phi_j
    tf: float

    def w(self, t: float) -> np.ndarray:
        return math.exp(self.tf - t) * self.profile

    def rhs(self) -> np.ndarray:
        """All-at-once right-hand side [M w(0) ; 0 ... ; load of f at every stage time]."""
        op = self.op
        v = np.zeros((op.nt + 1, op.nx))
        V = np.zeros((op.nt, op.s, op.nx))
        v[0] = op.Mmul(self.w(0.0))
        fc = math.pi ** 2 / 2.0 - 1.0
        for n in range(op.nt):
            for i in range(op.s):
                t = (n + op.c[i]) * op.tau
                V[n, i] = fc * math.exp(self.tf - t) * self.load_profile
        return op.join(v, V)

    def v_error(self, x: np.ndarray) -> float:
        op = self.op
        wv = np.asarray(x)[: op.n_v].reshape(op.nt + 1, op.nx)
        err = 0.0
        for n in range(op.nt + 1):
            exact = self.w(n * op.tau) + 1.0
            d = np.abs(wv[n] + 1.0 - exact)
            j = int(np.argmax(d))
            err = max(err, float(d[j] / abs(exact[j])))
        return err


def exact_solution_problem(disc: str, l: int, s: int, tf: float = T_FINAL, quad: int = 8) -> ExactSolutionProblem:
    if disc not in ("q1", "q2"):
        raise ValueError("the test problem is defined for Q1 and Q2 elements")
    n = level_nodes(disc, l)
    ns = (n, n)
    M, K = operators(ns, (LENGTH, LENGTH), disc)
    nt = time_steps(disc, l, s, tf)
    A, b, c = tableau("radau", s)
    op = AllAtOnce(K, M, tf / nt, nt, A, b, c)
    op.mass_interval = (q1_jacobi_interval if disc == "q1" else q2_jacobi_interval)(2)
    X = np.arange(1, n + 1) * (LENGTH / (n + 1))
    prof1 = np.sin(math.pi * X / 2.0)
    g1 = load_1d(disc, n, lambda Z: np.sin(math.pi * Z / 2.0), LENGTH, quad)
    return ExactSolutionProblem(disc, l, s, op, n, np.outer(prof1, prof1).ravel(), np.outer(g1, g1).ravel(), tf)
