"""Pins of the oracle's relaxed-product FGMRES (oracle/relaxed.py): the iteration-dependent matvec
precision of the paper's future-work paragraph, with the inexact-Krylov bound it cites."""
import numpy as np
import scipy.sparse as sp

import synth
from oracle.fgmres import fgmres
from oracle.precond import Preconditioner
from oracle.relaxed import U32, fgmres_relaxed, fp32_product, gamma
from oracle.solve import build


def _problem(ns=(9, 8), nt=4, s=2):
    op = build(ns, 1.0, nt, "radau", s)
    rhs = op.rhs(synth.random_vector(op.nx, 1), synth.random_vector(op.nx, 2))
    return op, rhs


def _precond(op, ns=(9, 8)):
    return Preconditioner(op, ns, inner_maxit=3, inner_tol=1e-3, omega=0.8)


def test_gamma_bounds_products_of_roundings():
    """Higham Lemma 3.1: a product of d factors (1 + delta_i), |delta_i| <= u, lies within
    gamma_d of 1; the worst case (1 + u)^d - 1 is below gamma_d, and gamma_d exceeds d u."""
    from fractions import Fraction
    u = Fraction(1, 2 ** 24)
    for d in (1, 2, 5, 24, 100):
        worst = (1 + u) ** d - 1
        assert float(worst) <= gamma(d) and gamma(d) > d * U32


def test_no_relaxation_and_exact_product_reproduce_fgmres():
    """ell = 0 never accepts an inexact product; an exact 'inexact' product (bound 0) is always
    accepted.  Both give the iterates of oracle.fgmres.fgmres bit for bit (restarts included)."""
    op, rhs = _problem()
    x0, k0, r0, ok0 = fgmres(op.matvec, _precond(op).apply, rhs, 1e-11, 3, 100)
    never = lambda z, allowed: (op.matvec(z) + 1.0, 1e-300)      # wrong, but never accepted at ell = 0
    x1, k1, r1, ok1 = fgmres_relaxed(op.matvec, never, _precond(op).apply, rhs, 1e-11, 3, 100, ell=0.0)
    log = []
    exact = lambda z, allowed: (op.matvec(z), 0.0)
    x2, k2, r2, ok2 = fgmres_relaxed(op.matvec, exact, _precond(op).apply, rhs, 1e-11, 3, 100, ell=1.0, log=log)
    assert ok0 and ok1 and ok2 and k0 == k1 == k2 and k0 > 3
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2) and r0 == r1 == r2
    assert all(e["relaxed"] for e in log if "relaxed" in e)


def test_worst_case_inexact_product_obeys_the_gap_bound():
    """Simoncini--Szyld: with ||f_k|| <= ell tol ||b|| / (m |g_k|) at every iteration, a cycle of j
    iterations ends with |r_true - |g|| <= ell tol ||b|| (j / m) / sigma_min(H).  Error of exactly
    the allowed norm in a random direction; the bound holds and is not vacuous."""
    op, rhs = _problem()
    rng = np.random.default_rng(5)

    def worst(z, allowed):
        f = rng.standard_normal(z.shape)
        return op.matvec(z) + allowed * f / np.linalg.norm(f), allowed

    tol, m, ell = 1e-6, 20, 1.0
    log = []
    x, k, rr, ok = fgmres_relaxed(op.matvec, worst, _precond(op).apply, rhs, tol, m, 100, ell=ell, log=log)
    ends = [e for e in log if "cycle_end" in e]
    bnorm = np.linalg.norm(rhs)
    assert ends
    for e in ends:
        bound = ell * tol * bnorm * (e["iterations"] / m) / e["sigma_min"]
        assert e["gap"] <= bound * (1 + 1e-8) + 1e-13 * bnorm, (e["gap"], bound)
    assert max(e["gap"] for e in ends) >= 1e-4 * ell * tol * bnorm / m       # the error shows
    # |y_k| <= |g_k| / sigma_min (the lemma the bound rests on), first cycle
    its = [e for e in log if "relaxed" in e][: ends[0]["iterations"]]
    g = [e0["allowed"] for e0 in its]                       # allowed_k = ell tol ||b|| / (m |g_k|)
    gk = [ell * tol * bnorm / (m * a) for a in g]
    for yk, gkk in zip(ends[0]["y"], gk):
        assert abs(yk) <= gkk / ends[0]["sigma_min"] * (1 + 1e-10)


def test_fp32_product_obeys_its_componentwise_bound():
    """|fl32(A z) - A z| <= gamma_d |A||z| entry by entry, on the all-at-once operator (which has
    cancellation: the bound is far above the error there) and on a nonnegative matrix and vector
    (no cancellation: the bound is within a small factor of the error, so it is not vacuous)."""
    op, _ = _problem(ns=(7, 6), nt=3, s=3)
    A = sp.csr_matrix(op.dense())
    d = int(np.diff(A.indptr).max()) + 2
    for seed in range(3):
        z = synth.random_vector(A.shape[1], 40 + seed)
        w, bound = fp32_product(A, z)
        err = np.abs(w - A @ z)
        assert np.all(err <= gamma(d) * (abs(A) @ np.abs(z)) + 1e-300)
        assert np.linalg.norm(w - A @ z) <= bound
    rng = np.random.default_rng(3)
    P = sp.random(400, 400, density=0.1, random_state=4, format="csr")
    z = rng.random(400)
    w, bound = fp32_product(P, z)
    obs = np.linalg.norm(w - P @ z)
    assert obs <= bound and obs >= bound / 200


def test_relaxed_solve_of_the_all_at_once_system():
    """The FP32 product inside the solve: late iterations (small |g_k|) take it, early ones the
    exact product; the TRUE residual reaches the tolerance and the solution matches the exact
    FGMRES solution to the tolerance's level."""
    ns, nt, s = (10, 9), 4, 2
    op = build(ns, 1.0, nt, "radau", s)
    rhs = op.rhs(synth.random_vector(op.nx, 3), synth.random_vector(op.nx, 4))
    A = sp.csr_matrix(op.dense())
    low = lambda z, allowed: fp32_product(A, z)
    log = []
    tol = 1e-10
    x, k, rr, ok = fgmres_relaxed(op.matvec, low, _precond(op, ns).apply, rhs, tol, 20, 100, ell=1.0, log=log)
    xe, ke, rre, oke = fgmres(op.matvec, _precond(op, ns).apply, rhs, tol, 20, 100)
    flags = [e["relaxed"] for e in log if "relaxed" in e]
    print(f"relaxed: {flags}")
    assert ok and rr <= tol and not flags[0] and any(flags)
    # once relaxed, later iterations of the cycle stay relaxed (|g_k| only falls; bounds similar)
    first = flags.index(True)
    assert all(flags[first:])
    assert np.linalg.norm(x - xe) <= 1e3 * tol * np.linalg.norm(xe)
