"""Pins of the oracle's split-preconditioned FGMRES (Algorithm 1 with P_L != I)."""
import numpy as np
import pytest

import synth
from oracle.fgmres import fgmres, fgmres_split
from oracle.precond import Preconditioner
from oracle.solve import build


def _identity(v):
    return np.array(v, dtype=np.float64, copy=True)


def _problem(ns=(9, 8), nt=4, s=2):
    op = build(ns, 1.0, nt, "radau", s)
    rhs = op.rhs(synth.random_vector(op.nx, 1), synth.random_vector(op.nx, 2))
    return op, rhs


def test_left_identity_reduces_to_right_preconditioned_fgmres():
    """P_L = I: the same iterates as the right-preconditioned solver, with an inexact (nonlinear)
    P_tilde on the right and restarts."""
    op, rhs = _problem()
    P1 = Preconditioner(op, (9, 8), inner_maxit=3, inner_tol=1e-3, omega=0.8)
    P2 = Preconditioner(op, (9, 8), inner_maxit=3, inner_tol=1e-3, omega=0.8)
    h1, h2 = [], []
    x1, k1, r1, ok1 = fgmres(op.matvec, P1.apply, rhs, 1e-11, 3, 100, history=h1)
    x2, k2, r2, ok2 = fgmres_split(op.matvec, _identity, P2.apply, rhs, 1e-11, 3, 100, history=h2)
    assert ok1 and ok2 and k1 == k2 and k1 > 3            # several restart cycles
    assert np.array_equal(x1, x2) and h1 == h2 and r1 == r2


@pytest.mark.parametrize("side", ["left", "right"])
def test_exact_preconditioner_converges_in_two_iterations_either_side(side):
    """Sec. 3: with exact blocks P^{-1} A (and A P^{-1}) has the single eigenvalue 1 and a minimal
    polynomial of degree 2, so GMRES converges in two iterations on either side."""
    op, rhs = _problem(nt=3, s=3)
    P = Preconditioner(op, (9, 8), exact=True)
    h = []
    if side == "left":
        x, k, r, ok = fgmres_split(op.matvec, P.apply, _identity, rhs, 1e-13, 20, 2, history=h)
    else:
        x, k, r, ok = fgmres_split(op.matvec, _identity, P.apply, rhs, 1e-13, 20, 2, history=h)
    assert h[0] > 1e-3 and h[1] < 1e-10 and k == 2          # two iterations, then rounding level
    xd = np.linalg.solve(op.dense(), rhs)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_left_preconditioning_by_A_itself_takes_one_iteration():
    op, rhs = _problem(ns=(5, 4), nt=2)
    lu = np.linalg.inv(op.dense())
    x, k, r, ok = fgmres_split(op.matvec, lambda v: lu @ v, _identity, rhs, 1e-12, 20, 5)
    assert ok and k == 1 and r <= 1e-12


def test_left_preconditioned_inexact_solve_reaches_the_solution():
    """Left preconditioning with the inexact P_tilde (the paper's parallel runs): the test is on the
    preconditioned residual; the solution still matches a dense solve."""
    op, rhs = _problem()
    P = Preconditioner(op, (9, 8), inner_maxit=5, inner_tol=1e-6, omega=0.8)
    x, k, r, ok = fgmres_split(op.matvec, P.apply, _identity, rhs, 1e-12, 20, 100)
    xd = np.linalg.solve(op.dense(), rhs)
    assert ok and np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
