"""Two-level MGRIT for S_tilde's time recurrence on the GPU (the parallel implementation of
Sec. 5) against the oracle's MGRIT (oracle.mgrit through oracle.precond with schur="mgrit",
one iteration, F-relaxation), element by element in FP64, and mixed-precision solves with it
against the exact all-at-once solution."""
import numpy as np
import pytest

import synth
from oracle.precond import Preconditioner
from oracle.fgmres import fgmres
from oracle.solve import build

from gpu_util import dev, host, rel_max, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def make(ns, nt, m, method="radau", s=2, prec="fp64", disc="fd", **kw):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make as tab
    dev()
    itol = kw.get("inner_tol", 1e-6)
    S = Solver(ns, 1.0, nt, tableau=tab(method, s), prec_P=prec, inner_maxit=3, inner_tol=itol, mg_cycles=3,
               mg_pre=2, mg_post=2, mg_omega=0.8, tol=kw.get("tol", 1e-10), disc=disc, mgrit_m=m)
    op = build(ns, 1.0, nt, method, s, disc=disc)
    P = (Preconditioner(op, ns, 3, itol, 3, 2, 2, 0.8, schur="mgrit", mgrit_m=m, mgrit_iters=1, mgrit_relax="F")
         if m > 0 else Preconditioner(op, ns, 3, itol, 3, 2, 2, 0.8))
    return S, op, P


# 2D grids with a cluster plan take the lock-step schedule (batched relaxation steps); 3D grids and
# 100 x 12 (no cluster plan) take the dataflow schedule over worker streams
CASES = [((24, 20), 8, 4, "radau", 3, "fd"), ((40, 36), 16, 8, "radau", 2, "fd"), ((33, 17), 6, 2, "gauss", 2, "fd"),
         ((7, 6, 5), 6, 3, "radau", 2, "fd"), ((10, 12), 4, 2, "radau", 2, "q1"), ((48, 40), 4, 4, "radau", 3, "fd"),
         ((100, 12), 8, 4, "radau", 2, "fd"), ((9, 8, 10), 12, 3, "gauss", 2, "fd"),
         # coarsening factors that do not divide nt: a shorter final interval (both schedules)
         ((40, 36), 16, 5, "radau", 2, "fd"), ((24, 20), 8, 3, "radau", 3, "fd"), ((100, 12), 10, 4, "radau", 2, "fd"),
         ((9, 8, 10), 12, 5, "gauss", 2, "fd"), ((10, 12), 7, 3, "radau", 2, "q1")]


@pytest.mark.parametrize("ns,nt,m,method,s,disc", CASES)
def test_mgrit_precond_matches_oracle(ns, nt, m, method, s, disc):
    S, op, P = make(ns, nt, m, method, s, disc=disc)
    r = synth.random_vector(op.n_st, 160)
    z = host(S.precond_apply(to_dev(r), zeros(op.n_st)))
    assert rel_max(z, P.apply(r)) <= 1e-11
    zt = host(S.precond_apply(to_dev(r), zeros(op.n_st), transpose=True))
    assert rel_max(zt, P.apply_T(r)) <= 1e-11


def test_mgrit_with_one_interval_is_the_substitution():
    """m = nt: one coarse interval, the F-relaxation alone runs the whole recurrence exactly."""
    ns, nt, s = (40, 36), 6, 3
    S, op, _ = make(ns, nt, nt, "radau", s)
    S0, _, _ = make(ns, nt, 0, "radau", s)
    r = to_dev(synth.random_vector(op.n_st, 161))
    z = host(S.precond_apply(r, zeros(op.n_st)))
    z0 = host(S0.precond_apply(r, zeros(op.n_st)))
    assert rel_max(z, z0) <= 1e-12
    zt = host(S.precond_apply(r, zeros(op.n_st), transpose=True))
    zt0 = host(S0.precond_apply(r, zeros(op.n_st), transpose=True))
    assert rel_max(zt, zt0) <= 1e-12


def test_mgrit_fp64_solve_matches_oracle_iterations():
    ns, nt, m, s = (32, 32), 16, 4, 3
    S, op, P = make(ns, nt, m, "radau", s, tol=1e-10)
    u0 = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(7, "u0"))
    f = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(7, "f"))
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(op.n_st))
    xr, its, rr, ok = fgmres(op.matvec, P.apply, op.rhs(u0, f), 1e-10, 20, 100)
    print(f"MGRIT FP64: GPU its {info.outer_its} oracle its {its}")
    assert info.converged and ok and info.outer_its == its
    assert np.linalg.norm(host(x) - xr) <= 1e-10 * np.linalg.norm(xr)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mgrit_mixed_solve_against_exact_solution(prec):
    from oracle import spectral
    from oracle.tableau import tableau
    ns, nt, m, s = (64, 64), 32, 8, 3
    S, op, _ = make(ns, nt, m, "radau", s, prec=prec, tol=1e-8, inner_tol=1e-3)
    u0 = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(8, "u0"))
    f = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(8, "f"))
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(op.n_st))
    A, b, _ = tableau("radau", s)
    exact = spectral.solve(ns, op.tau, nt, A, b, op.rhs(u0, f))
    err = np.linalg.norm(host(x) - exact) / np.linalg.norm(exact)
    print(f"MGRIT {prec}: outer its {info.outer_its}, error vs the exact solution {err:.2e}")
    assert info.converged and err <= 1e-8


def test_schedule_autotuner_returns_a_timed_candidate():
    from paper_2609_16863_gb300 import tune_mgrit, radau_iia
    dev()
    best, times = tune_mgrit((48, 40), 1.0, 16, tableau=radau_iia(2), prec_P="fp32", inner_maxit=3, inner_tol=1e-3)
    assert set(times) == {0, 4, 6, 8} and best in times and all(t > 0 for t in times.values())
    fastest = min(times, key=times.get)
    # the fastest MGRIT candidate, unless it beats the substitution by 10% or less
    assert best == (fastest if fastest == 0 or times[fastest] <= 0.9 * times[0] else 0)
