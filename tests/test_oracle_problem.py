"""Pins of the Q2 elements and of the paper's exact-solution test problem (Sec. 5.1, Table 2)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.aao import dof_count
from oracle.operators import _q2_1d, q2_matrices
from oracle.problems import exact_solution_problem, load_1d, level_nodes, time_steps
from oracle.sequential import sequential_rk, sequential_solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_verror.txt")
TABLE = {(int(r[0]), int(r[1])): (float(r[2]), float(r[3]))
         for r in (ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#"))}


def test_q2_element_matrices_integrate_quadratics_exactly():
    """u = X (L - X) lies in the interior Q2 space, so M u is its load vector int u phi_j and, by
    parts, K u is the load of -u'' = 2; both by Gauss quadrature exact for these integrands."""
    n, L = 11, 2.0
    X = np.arange(1, n + 1) * (L / (n + 1))
    M, K = _q2_1d(n, L / (n + 1))
    u = X * (L - X)
    assert np.abs(M @ u - load_1d("q2", n, lambda Z: Z * (L - Z), L, 3)).max() < 1e-14
    assert np.abs(K @ u - load_1d("q2", n, lambda Z: 2.0 + 0.0 * Z, L, 3)).max() < 1e-13
    assert abs(u @ M @ u - L ** 5 / 30) < 1e-13                 # int u^2
    assert abs(u @ K @ u - L ** 3 / 3) < 1e-12                  # int u'^2


def test_q2_2d_matrices_symmetric_positive_and_tensor():
    M, K = q2_matrices((7, 5), (2.0, 1.0))
    assert abs(M - M.T).max() == 0.0 and abs(K - K.T).max() == 0.0
    assert np.linalg.eigvalsh(M.toarray()).min() > 0 and np.linalg.eigvalsh(K.toarray()).min() > 0
    Mx, Kx = _q2_1d(7, 2.0 / 8)
    My, Ky = _q2_1d(5, 1.0 / 6)
    assert abs(K - (sp.kron(My, Kx) + sp.kron(Ky, Mx))).max() < 1e-12


def test_dof_and_time_steps_match_table2():
    rows = {(2, 3): (931, 5625), (3, 5): (27869, 178605), (5, 7): (596773, 3186225)}
    for (s, l), (q1, q2) in rows.items():
        assert dof_count(level_nodes("q1", l) ** 2, time_steps("q1", l, s), s) == q1
        assert dof_count(level_nodes("q2", l) ** 2, time_steps("q2", l, s), s) == q2


def test_sequential_solve_matches_time_stepping():
    P = exact_solution_problem("q1", 3, 2)
    op = P.op
    f = np.random.default_rng(0).standard_normal(op.nt * op.s * op.nx)
    u0 = P.w(0.0)
    ref = sequential_rk(op, u0, f, f_time_dep=True)
    assert np.abs(sequential_solve(op, op.rhs(u0, f, f_time_dep=True)) - ref).max() <= 1e-12 * np.abs(ref).max()


# cells whose printed error is set by the discretisation: errors below 1e-7 sit at the level of the
# paper's outer tolerance 1e-8 and are left out, as are the largest grids (time)
CELLS = [(disc, s, l) for s in (2, 3, 4, 5) for l in (3, 4, 5, 6) for disc in ("q1", "q2")
         if TABLE[(s, l)][disc == "q2"] >= 1e-7 and not (disc == "q2" and l == 6)]


@pytest.mark.parametrize("disc,s,l", CELLS)
def test_discretisation_error_matches_table2(disc, s, l):
    """The oracle's Q2 discrete solution reproduces the printed v_error within 25% (within 1% where
    the time error is negligible, s >= 4); Q1 comes out 7-35% above the printed values at every
    level (same order in h; the paper's Q1 source or initial-data treatment is not stated)."""
    P = exact_solution_problem(disc, l, s)
    e = P.v_error(sequential_solve(P.op, P.rhs()))
    ratio = e / TABLE[(s, l)][disc == "q2"]
    if disc == "q2":
        assert (0.99 <= ratio <= 1.01) if s >= 4 else (0.95 <= ratio <= 1.25), ratio
    else:
        assert 1.0 <= ratio <= 1.4, ratio


@pytest.mark.parametrize("disc,s,order", [("q1", 5, 2), ("q2", 5, 3)])
def test_convergence_order_in_h(disc, s, order):
    """Error ratios between levels l = 3, 4, 5: at least 2^order * 0.85 (Q1 nodal order 2; Q2 order
    3, nodal superconvergence allowed), with s = 5 so that the time error is negligible."""
    errs = []
    for l in (3, 4, 5):
        P = exact_solution_problem(disc, l, s)
        errs.append(P.v_error(sequential_solve(P.op, P.rhs())))
    for a, b in zip(errs, errs[1:]):
        assert a / b >= 0.85 * 2 ** order, (errs, order)


def test_chebyshev_mass_inverse_bound_q2():
    """||e_k||_M <= ||e_0||_M / T_k(sigma) with the Q2 interval [1/4, 25/16] (element-by-element
    bound of D^{-1} M), on the assembled 2D Q2 mass matrix."""
    import scipy.sparse.linalg as spla
    from oracle.operators import q2_jacobi_interval
    from oracle.precond import chebyshev_jacobi
    M, _ = q2_matrices((15, 13), (1.0, 2.0))
    A = M.toarray()
    ev = np.linalg.eigvals(np.linalg.solve(np.diag(np.diag(A)), A)).real
    lo, hi = q2_jacobi_interval(2)
    assert lo <= ev.min() and ev.max() <= hi * (1 + 1e-12)
    g = np.random.default_rng(2).standard_normal(M.shape[0])
    x = spla.spsolve(M.tocsc(), g)
    sig = (hi + lo) / (hi - lo)
    for k in (5, 10, 20):
        e = x - chebyshev_jacobi(M, g, k, lo, hi)
        ratio = np.sqrt(e @ (M @ e) / (x @ (M @ x)))
        assert ratio <= 1.0 / np.cosh(k * np.arccosh(sig)) * 1.01


@pytest.mark.parametrize("disc,s,l", [("q2", 2, 3), ("q1", 3, 4)])
def test_preconditioned_solve_of_the_exact_solution_problem(disc, s, l):
    """FGMRES with P_tilde (multigrid, Chebyshev M^{-1} with the element's interval) on the paper's
    problem reaches the direct solution."""
    from oracle.fgmres import fgmres
    from oracle.precond import Preconditioner
    P = exact_solution_problem(disc, l, s)
    pre = Preconditioner(P.op, (P.n, P.n), inner_maxit=5, inner_tol=1e-6, omega=0.8)
    x, its, rr, ok = fgmres(P.op.matvec, pre.apply, P.rhs(), 1e-12, 20, 100)
    ref = sequential_solve(P.op, P.rhs())
    assert ok and np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    assert abs(P.v_error(x) - P.v_error(ref)) <= 1e-6 * P.v_error(ref)
