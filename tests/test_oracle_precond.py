"""Pins of the oracle's preconditioner pieces (Sec. 3, Sec. 5, Fig. 1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle.multigrid import Hierarchy, interp_1d, level_sizes
from oracle.precond import Preconditioner, chebyshev_jacobi, gmres_fixed
from oracle.solve import OracleOptions, build, solve
from oracle.operators import q1_matrices


def test_exact_preconditioner_two_iterations():
    # Sec. 3: sigma(P^{-1} A) = {1}, minimal polynomial of degree 2
    for ns, nt, method, s in (((10, 10), 5, "radau", 3), ((5, 5, 5), 2, "gauss", 2)):
        op = build(ns, 1.0, nt, method, s)
        rhs = op.rhs(synth.random_vector(op.nx, 1), synth.random_vector(op.nx, 2))
        r = solve(op, ns, rhs, OracleOptions(tol=1e-15, maxit=2, exact=True))
        assert r.history[0] > 1e-3          # one iteration is not enough
        assert r.history[1] < 1e-10         # two are, up to rounding


def test_exact_schur_propagates_initial_data():
    # with exact Theta_tilde, S^{-1} [u0; 0; ...] is unforced RK propagation of u0
    ns, nt, s = (9, 9), 6, 3
    op = build(ns, 1.0, nt, "radau", s)
    P = Preconditioner(op, ns, exact=True)
    u0 = synth.random_vector(op.nx, 3)
    r = np.zeros(op.n_st)
    r[: op.nx] = u0
    z = P.apply(r)
    from oracle.sequential import sequential_rk
    xs = sequential_rk(op, u0, np.zeros(op.nx))
    zv = z[: op.n_v]
    assert np.linalg.norm(zv - xs[: op.n_v]) <= 1e-12 * np.linalg.norm(xs[: op.n_v])


def test_exact_preconditioner_transpose_is_adjoint():
    ns, nt = (6, 5), 3
    op = build(ns, 1.0, nt, "radau", 2)
    P = Preconditioner(op, ns, exact=True)
    a = synth.random_vector(op.n_st, 1)
    b = synth.random_vector(op.n_st, 2)
    lhs = P.apply(a) @ b
    rhs = a @ P.apply_T(b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_pint_matches_dense_block_triangular():
    ns, nt, s = (5, 6), 2, 3
    op = build(ns, 1.0, nt, "radau", s)
    P = Preconditioner(op, ns, exact=True)
    K = op.K.toarray()
    Pint = np.kron(np.eye(s), np.eye(op.nx)) + op.tau * np.kron(P.L @ np.diag(P.D), K)
    r = synth.random_vector(s * op.nx, 4)
    assert np.allclose(P.pint_apply(r), np.linalg.solve(Pint, r), rtol=0, atol=1e-12 * np.abs(r).max())
    assert np.allclose(P.pint_apply_T(r), np.linalg.solve(Pint.T, r), rtol=0, atol=1e-12 * np.abs(r).max())


def test_rana_backward_euler_is_exact():
    # s = 1: P_int = Theta_hat, so one inner iteration solves it exactly
    ns = (7, 7)
    op = build(ns, 1.0, 4, "radau", 1)
    P = Preconditioner(op, ns, inner_maxit=5, inner_tol=1e-14, exact=False)
    P.shifted_solve = lambda i, r: spla.spsolve(P.shifted[i].tocsc(), r)
    r = synth.random_vector(op.nx, 5)
    z, its = gmres_fixed(P.theta_apply, P.pint_apply, r, 5, 1e-14)
    assert its == 1
    assert np.allclose(z, spla.spsolve(op.theta_hat().tocsc(), r), rtol=1e-12, atol=0)


def test_inner_gmres_full_dimension_is_exact():
    ns = (3, 3)
    op = build(ns, 1.0, 2, "radau", 2)
    P = Preconditioner(op, ns)
    r = synth.random_vector(2 * op.nx, 6)
    z, its = gmres_fixed(P.theta_apply, lambda v: v, r, 2 * op.nx, 0.0)
    assert np.allclose(z, np.linalg.solve(op.theta_hat().toarray(), r), rtol=1e-10, atol=0)


def test_gmres_residual_estimate_is_true_residual():
    ns = (8, 8)
    op = build(ns, 1.0, 2, "radau", 3)
    P = Preconditioner(op, ns)
    r = synth.random_vector(3 * op.nx, 7)
    Th = op.theta_hat()
    for k in (1, 2, 3):
        z, its = gmres_fixed(P.theta_apply, P.pint_apply, r, k, 0.0)
        assert its == k
    # monotone decrease of the true residual with more iterations
    res = [np.linalg.norm(r - Th @ gmres_fixed(P.theta_apply, P.pint_apply, r, k, 0.0)[0]) for k in (1, 2, 3, 4)]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(3))


# ---------------- multigrid ----------------

def test_interp_1d_small():
    P4 = interp_1d(4).toarray()
    assert np.array_equal(P4, [[0.5, 0], [1, 0], [0.5, 0.5], [0, 1]])
    P5 = interp_1d(5).toarray()
    assert np.array_equal(P5, [[0.5, 0], [1, 0], [0.5, 0.5], [0, 1], [0, 0.5]])
    # coarsening stops at the first level with <= 256 unknowns, or when an axis cannot be halved
    assert level_sizes((32, 32)) == [(32, 32), (16, 16)]
    assert level_sizes((256, 256))[-1] == (16, 16) and len(level_sizes((256, 256))) == 5
    assert level_sizes((96,) * 3) == [(96,) * 3, (48,) * 3, (24,) * 3, (12,) * 3, (6,) * 3]
    assert level_sizes((300, 4)) == [(300, 4), (150, 2)]
    assert level_sizes((15, 17)) == [(15, 17)]


def test_galerkin_closed_form():
    # constant coefficients, N = 2^k - 1: P^T (I (x) K1 + K1 (x) I) P has the interior
    # stencil (P1^T K1 P1) (x) (P1^T P1) + (P1^T P1) (x) (P1^T K1 P1) with
    # P1^T K1 P1 = (1/(2 h^2)) tridiag(-1, 2, -1) and P1^T P1 = tridiag(1/4, 3/2, 1/4).
    N, c = 31, 0.3
    ns = (N, N)
    op = build(ns, 1.0, 1, "radau", 1)
    A0 = (sp.identity(N * N) + c * op.K).tocsr()
    H = Hierarchy(A0, ns)
    Ac = H.A[1].toarray().reshape(15, 15, 15, 15)
    h = 1.0 / 32
    k1 = np.array([-1.0, 2.0, -1.0]) / (2 * h * h)
    m1 = np.array([0.25, 1.5, 0.25])
    sten = np.outer(m1, m1) + c * (np.outer(k1, m1) + np.outer(m1, k1))
    assert np.allclose(Ac[7, 7, 6:9, 6:9], sten, rtol=1e-13, atol=0)


def test_vcycle_symmetric_and_contracting():
    for ns in ((32, 32), (12, 12, 12), (20, 20)):
        op = build(ns, 1.0, 32, "radau", 3)
        P = Preconditioner(op, ns)
        H = P.mg[0]
        x = synth.random_vector(op.nx, 1)
        y = synth.random_vector(op.nx, 2)
        Bx = H.solve(x, 1)
        By = H.solve(y, 1)
        assert abs(y @ Bx - x @ By) <= 1e-12 * abs(y @ Bx)
        # contraction of the error propagator I - B A over repeated cycles
        A = P.shifted[0]
        e = synth.random_vector(op.nx, 3)
        for _ in range(4):
            e_new = e - H.solve(A @ e, 1)
            fac = np.linalg.norm(e_new) / np.linalg.norm(e)
            e = e_new
        assert fac <= 0.2


def test_coarsest_level_is_exact():
    ns = (3, 3)                      # a single level: the V-cycle is the direct solve
    op = build(ns, 1.0, 1, "radau", 1)
    A0 = (sp.identity(9) + 0.1 * op.K).tocsr()
    H = Hierarchy(A0, ns)
    assert H.nlevels == 1
    b = synth.random_vector(9, 1)
    assert np.allclose(H.solve(b, 1), np.linalg.solve(A0.toarray(), b), rtol=1e-14, atol=0)


def test_chebyshev_mass_inverse_bound():
    # The Chebyshev error polynomial has max 1/T_k(sigma) on the D^{-1}M spectrum, and
    # D^{-1}M is self-adjoint in the M inner product, so ||e_k||_M <= ||e_0||_M / T_k(sigma)
    # with the Q1 interval [1/4, 9/4] (sigma = 5/4).
    M, _ = q1_matrices((15, 15))
    g = synth.random_vector(M.shape[0], 1)
    x = spla.spsolve(M.tocsc(), g)
    lo, hi = 0.25, 2.25
    sig = (hi + lo) / (hi - lo)
    D = M.diagonal()
    for k in (5, 10, 20):
        xk = chebyshev_jacobi(M, g, k, lo, hi)
        Tk = np.cosh(k * np.arccosh(sig))
        # error in the M-norm, bounded by 2/T_k times the initial error
        e, e0 = x - xk, x
        ratio = np.sqrt(e @ (M @ e) / (e0 @ (M @ e0)))
        assert ratio <= 1.0 / Tk * 1.01
