"""Pins of the oracle's two-level MGRIT for S_tilde's time recurrence (Sec. 5, parallel
implementation; algorithm of Falgout et al. 2014)."""
import math

import numpy as np
import pytest

import synth
from oracle import mgrit
from oracle.precond import Preconditioner
from oracle.solve import build

NS = (17, 17)          # two multigrid levels


def _precond(nt, m, s=2, exact=False, **kw):
    op = build(NS, 1.0, nt, "radau", s)
    P = Preconditioner(op, NS, inner_maxit=3, inner_tol=0.0, mg_cycles=3, nu1=2, nu2=2, omega=0.8,
                       exact=exact, schur="mgrit", mgrit_m=m, **kw)
    return op, P


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("m,k,relax", [(4, 1, "F"), (4, 1, "FCF"), (3, 2, "F"), (3, 2, "FCF"), (2, 1, "FCF"),
                                       (6, 1, "FCF"), (5, 1, "F"), (5, 2, "FCF"), (7, 2, "F"), (10, 1, "F")])
def test_mgrit_exact_prefix(m, k, relax):
    """After k iterations the first (k+1)m (F) or (2k+1)m (FCF) points equal sequential
    substitution, whatever the coarse propagator; the next C-point does not.  m = 5, 7, 10 do not
    divide nt = 24: the steps after the last C-point form a shorter final interval."""
    nt = 24
    op, P = _precond(nt, m)
    w = np.stack([synth.random_vector(op.nx, 100 + n) for n in range(nt + 1)])
    u = mgrit.two_level(P.schur_step, P.coarse.schur_step, w, m, k, relax)
    ref = mgrit.sequential(P.schur_step, w)
    p = min(((2 * k + 1) if relax == "FCF" else (k + 1)) * m, nt + 1)
    assert _rel(u[:p], ref[:p]) <= 1e-12
    if p <= nt:        # the next C-point is off by more than rounding (MGRIT converges fast here)
        assert np.abs(u[p] - ref[p]).max() > 1e-10 * np.abs(ref[p]).max()


@pytest.mark.parametrize("relax,m", [("F", 4), ("FCF", 4), ("F", 5), ("FCF", 7)])
def test_mgrit_ideal_coarse_propagator_converges_in_one_iteration(relax, m):
    """For a linear step Phi (exact stage solves) and Phi_c = Phi^m, one iteration is exact (for
    m = 5, 7 the shorter final interval included)."""
    nt = 24
    op, P = _precond(nt, m, exact=True)

    def phi_m(e):
        for _ in range(m):
            e = P.schur_step(e)
        return e

    w = np.stack([synth.random_vector(op.nx, 200 + n) for n in range(nt + 1)])
    u = mgrit.two_level(P.schur_step, phi_m, w, m, 1, relax)
    assert _rel(u, mgrit.sequential(P.schur_step, w)) <= 1e-12
    # the rediscretised coarse step is not ideal: one iteration is then only approximate
    u2 = mgrit.two_level(P.schur_step, P.coarse.schur_step, w, m, 1, relax)
    assert _rel(u2, mgrit.sequential(P.schur_step, w)) > 1e-8


def R_radau2(z):
    """Stability function of Radau IIA s=2 (Hairer & Wanner), a (1,2) Pade form."""
    return (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)


@pytest.mark.parametrize("mode", [(1, 1), (2, 3), (7, 4)])
def test_fine_and_coarse_steps_on_eigenmodes(mode):
    """With exact stage solves the S_tilde step maps a sine eigenmode phi (K phi = lambda phi) to
    R(-tau lambda) phi, and the coarse step to R(-m tau lambda) phi."""
    nt, m = 16, 4
    op, P = _precond(nt, m, exact=True)
    N = NS[0]
    h = 1.0 / (N + 1)
    k, l = mode
    lam = 4 / h ** 2 * (math.sin(k * math.pi * h / 2) ** 2 + math.sin(l * math.pi * h / 2) ** 2)
    phi = synth.sine_field(NS, [(k, l)])
    assert np.abs(op.K @ phi - lam * phi).max() <= 1e-10 * lam
    tau = 1.0 / nt
    assert _rel(P.schur_step(phi), R_radau2(-tau * lam) * phi) <= 1e-12
    assert _rel(P.coarse.schur_step(phi), R_radau2(-m * tau * lam) * phi) <= 1e-12
    # the backward (transposed) step is the same map for the symmetric FD operator
    assert _rel(P.coarse.schur_step_T(phi), R_radau2(-m * tau * lam) * phi) <= 1e-12


def test_mgrit_preconditioner_equals_substitution_with_enough_iterations():
    """k >= (nc - 1)/2 FCF iterations make P_tilde (and P_tilde^T) with MGRIT equal to the
    sequential one."""
    nt, m = 8, 2
    op, P = _precond(nt, m, s=3, mgrit_iters=2)
    Pseq = Preconditioner(op, NS, inner_maxit=3, inner_tol=0.0, mg_cycles=3, nu1=2, nu2=2, omega=0.8)
    r = synth.random_vector(op.n_st, 7)
    assert _rel(P.apply(r), Pseq.apply(r)) <= 1e-12
    assert _rel(P.apply_T(r), Pseq.apply_T(r)) <= 1e-12


def test_mgrit_preconditioned_solve_reaches_the_solution():
    """P_tilde only changes the path: FGMRES with one MGRIT iteration in S_tilde still converges
    to the solution of the all-at-once system."""
    from oracle.fgmres import fgmres
    nt, m = 4, 2
    op, P = _precond(nt, m, s=2)
    rhs = op.rhs(synth.random_vector(op.nx, 1), synth.random_vector(op.nx, 2))
    x, its, rr, ok = fgmres(op.matvec, P.apply, rhs, 1e-11, 20, 100)
    assert ok and rr <= 1e-11
    xd = np.linalg.solve(op.dense(), rhs)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_mgrit_rejects_bad_parameters():
    w = np.zeros((9, 4))
    with pytest.raises(ValueError):
        mgrit.two_level(lambda z: z, lambda z: z, w, 9, 1)          # m beyond the 8 steps
    with pytest.raises(ValueError):
        mgrit.two_level(lambda z: z, lambda z: z, w, 0, 1)
    with pytest.raises(ValueError):
        mgrit.two_level(lambda z: z, lambda z: z, w, 2, 1, "C")
    op = build(NS, 1.0, 6, "radau", 2)
    with pytest.raises(ValueError):
        Preconditioner(op, NS, schur="mgrit", mgrit_m=7)
    with pytest.raises(ValueError):                                 # three levels: 2^2 does not divide 6
        Preconditioner(op, NS, schur="mgrit", mgrit_m=2, mgrit_levels=3)


@pytest.mark.parametrize("relax,iters", [("FCF", 1), ("F", 2)])
def test_multilevel_with_two_levels_is_two_level(relax, iters):
    nt, m = 24, 4
    op, P = _precond(nt, m)
    w = np.stack([synth.random_vector(op.nx, 300 + n) for n in range(nt + 1)])
    a = mgrit.two_level(P.schur_step, P.coarse.schur_step, w, m, iters, relax)
    b = mgrit.multilevel([P.schur_step, P.coarse.schur_step], w, m, iters, relax)
    assert np.array_equal(a, b)


def test_three_levels_with_ideal_propagators_converge_in_one_cycle():
    """Linear Phi (exact stage solves), level propagators Phi^m and Phi^(m^2): one V-cycle is exact."""
    nt, m = 18, 3
    op, P = _precond(nt, m, exact=True)

    def power(k):
        def f(e):
            for _ in range(k):
                e = P.schur_step(e)
            return e
        return f

    w = np.stack([synth.random_vector(op.nx, 400 + n) for n in range(nt + 1)])
    u = mgrit.multilevel([P.schur_step, power(m), power(m * m)], w, m, 1, "F")
    assert _rel(u, mgrit.sequential(P.schur_step, w)) <= 1e-12


def test_three_level_preconditioner_converges_to_substitution():
    """Three levels with steps tau, 3 tau, 9 tau (re-discretised): V-cycles contract towards the
    substitution, and P_tilde / P_tilde^T with enough cycles equal the sequential ones."""
    nt, m = 18, 3
    op, P = _precond(nt, m, s=2, mgrit_levels=3)
    w = np.stack([synth.random_vector(op.nx, 500 + n) for n in range(nt + 1)])
    phis = [P.schur_step] + [c.schur_step for c in P.coarser]
    ref = mgrit.sequential(P.schur_step, w)
    errs = [_rel(mgrit.multilevel(phis, w, m, k, "FCF"), ref) for k in (1, 2, 3)]
    assert errs[0] < 1e-2 and errs[1] < 0.1 * errs[0] and errs[2] < 0.1 * errs[1]
    P9 = Preconditioner(op, NS, inner_maxit=3, inner_tol=0.0, mg_cycles=3, nu1=2, nu2=2, omega=0.8,
                        schur="mgrit", mgrit_m=m, mgrit_levels=3, mgrit_iters=4)
    Pseq = Preconditioner(op, NS, inner_maxit=3, inner_tol=0.0, mg_cycles=3, nu1=2, nu2=2, omega=0.8)
    r = synth.random_vector(op.n_st, 8)
    assert _rel(P9.apply(r), Pseq.apply(r)) <= 1e-9
    assert _rel(P9.apply_T(r), Pseq.apply_T(r)) <= 1e-9


@pytest.mark.parametrize("levels", [2, 3])
def test_mgrit_transposed_preconditioner_in_an_adjoint_solve(levels):
    """FGMRES on A^T with P_tilde^T using MGRIT (two or three levels) reaches the dense transposed
    solution: MGRIT changes only the path."""
    from oracle.fgmres import fgmres
    nt, m = 9, 3
    op, P = _precond(nt, m, s=2, mgrit_levels=levels)
    g = synth.random_vector(op.n_st, 12)
    lam, its, rr, ok = fgmres(op.rmatvec, P.apply_T, g, 1e-11, 20, 100)
    ref = np.linalg.solve(op.dense().T, g)
    assert ok and np.linalg.norm(lam - ref) <= 1e-8 * np.linalg.norm(ref)
