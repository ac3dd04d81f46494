"""Pins of the oracle's spatial operators and all-at-once operator (Sec. 2)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.aao import AllAtOnce, dof_count
from oracle.operators import q1_matrices, stiffness_fd
from oracle.solve import OracleOptions, build, solve
from oracle.tableau import tableau

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_dof.txt")


def _nt_rule(l, s, q_fe, tf=2.0):
    # Sec. 5: n_t the smallest integer with tau = tf/n_t <= h^(q_FE/q_RK), h = 2^(1-l),
    # q_RK = 2s - 1 for Radau IIA
    h = 2.0 ** (1 - l)
    return math.ceil(tf / h ** (q_fe / (2 * s - 1)) - 1e-9)


def test_dof_counts_table2():
    rows = [list(map(int, ln.split())) for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 20
    for s, l, dof_q1, dof_q2 in rows:
        nx_q1 = (2 ** l - 1) ** 2
        nx_q2 = (2 ** (l + 1) - 1) ** 2
        assert dof_count(nx_q1, _nt_rule(l, s, 2), s) == dof_q1
        assert dof_count(nx_q2, _nt_rule(l, s, 3), s) == dof_q2


def test_dof_counts_parallel_cases():
    """The parallel test cases' printed DoF: n_x (1 + n_t (s + 1)) less one, for all three cases
    (an off-by-one in the printed counts; Table 2's counts match the formula exactly)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "parallel_dof.txt")
    rows = [list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for case, s, nx, nt, printed in rows:
        assert dof_count(nx, nt, s) == printed + 1, case
        # the operator's own layout count, per spatial unknown
        one = AllAtOnce(sp.identity(1, format="csr"), None, 1.0, nt, np.eye(s), np.ones(s) / s, np.ones(s))
        assert one.n_st * nx == dof_count(nx, nt, s)


def test_nst_matches_dof_count():
    op = build((5, 4), 1.0, 3, "radau", 3)
    assert op.n_st == dof_count(20, 3, 3)


def _lap1d(n, h):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h ** 2


@pytest.mark.parametrize("ns", [(4, 4), (5, 3), (3, 4, 5)])
def test_fd_stiffness_is_kron_laplacian(ns):
    hs = [1.0 / (n + 1) for n in ns]
    d = len(ns)
    I = [sp.identity(n) for n in ns]
    Kref = None
    for a in range(d):
        facs = [(_lap1d(ns[b], hs[b]) if b == a else I[b]) for b in reversed(range(d))]
        term = facs[0]
        for F in facs[1:]:
            term = sp.kron(term, F)
        Kref = term if Kref is None else Kref + term
    K = stiffness_fd(ns)
    assert abs(K - Kref).max() < 1e-9 * abs(Kref).max()


def test_fd_stiffness_variable_kappa():
    ns = (6, 5)
    rng = np.random.default_rng(1)
    kap = np.exp(rng.standard_normal((ns[1] + 2) * (ns[0] + 2)))
    K = stiffness_fd(ns, kappa=kap)
    assert abs(K - K.T).max() == 0.0
    # constant kappa = 3 scales the Laplacian
    K3 = stiffness_fd(ns, kappa=np.full_like(kap, 3.0))
    assert abs(K3 - 3.0 * stiffness_fd(ns)).max() < 1e-10
    # energy: u^T K u = sum over faces kappa_f (u_P - u_nb)^2 / h^2 (brute force)
    u = rng.standard_normal(ns[0] * ns[1])
    U = np.zeros((ns[1] + 2, ns[0] + 2)); U[1:-1, 1:-1] = u.reshape(ns[1], ns[0])
    Kp = kap.reshape(ns[1] + 2, ns[0] + 2)
    hx, hy = 1 / (ns[0] + 1), 1 / (ns[1] + 1)
    E = 0.0     # every pair of adjacent nodes; boundary values are 0
    for j in range(ns[1] + 2):
        for i in range(ns[0] + 2):
            for (dj, di, h) in ((0, 1, hx), (1, 0, hy)):
                jj, ii = j + dj, i + di
                if jj > ns[1] + 1 or ii > ns[0] + 1:
                    continue
                kf = 0.5 * (Kp[j, i] + Kp[jj, ii])
                E += kf * (U[j, i] - U[jj, ii]) ** 2 / h ** 2
    assert abs(u @ (K @ u) - E) < 1e-10 * E


def test_q1_mass_rows_and_jacobi_interval():
    ns = (7, 7)
    M, K = q1_matrices(ns)
    h = 1.0 / 8
    # interior rows away from the boundary integrate the hat function: h^2
    Md = M.toarray().reshape(7, 7, 7, 7)
    assert abs(Md[3, 3].sum() - h * h) < 1e-15
    # K annihilates linear functions in the interior (row sums of interior rows vanish)
    Kd = K.toarray().reshape(7, 7, 7, 7)
    assert abs(Kd[3, 3].sum()) < 1e-12
    ev = np.linalg.eigvals(np.diag(1 / M.diagonal()) @ M.toarray()).real
    assert ev.min() >= 0.25 - 1e-12 and ev.max() <= 2.25 + 1e-12


CASES = [((3, 3), 1, "radau", 1), ((3, 4), 3, "radau", 2), ((4, 3), 3, "radau", 3),
         ((3, 3, 3), 1, "gauss", 2), ((3, 3, 4), 3, "radau", 3), ((5, 5), 3, "radau", 3)]


@pytest.mark.parametrize("ns,nt,method,s", CASES)
def test_matvec_matches_dense_kronecker(ns, nt, method, s):
    op = build(ns, 0.7, nt, method, s)
    Ad = op.dense()
    x = synth.random_vector(op.n_st, 5)
    y = op.matvec(x)
    assert np.abs(y - Ad @ x).max() <= 1e-12 * np.abs(Ad @ x).max()
    assert np.abs(op.rmatvec(x) - Ad.T @ x).max() <= 1e-12 * np.abs(Ad.T @ x).max()


def test_matvec_q1_matches_dense():
    op = build((3, 4), 0.5, 2, "radau", 2, disc="q1")
    Ad = op.dense()
    x = synth.random_vector(op.n_st, 6)
    assert np.abs(op.matvec(x) - Ad @ x).max() <= 1e-12 * np.abs(Ad @ x).max()


@pytest.mark.parametrize("ns,nt,method,s", CASES)
def test_fgmres_solution_equals_dense_lu(ns, nt, method, s):
    op = build(ns, 0.7, nt, method, s)
    u0 = synth.random_vector(op.nx, 7)
    f = synth.random_vector(op.nx, 8)
    rhs = op.rhs(u0, f)
    x_lu = np.linalg.solve(op.dense(), rhs)
    r = solve(op, ns, rhs, OracleOptions(tol=1e-13))
    assert r.converged
    assert np.linalg.norm(r.x - x_lu) <= 1e-12 * np.linalg.norm(x_lu)


def test_rhs_layout():
    op = build((3, 3), 1.0, 2, "radau", 2)
    u0 = np.arange(9.0)
    f = np.ones(9)
    r = op.rhs(u0, f)
    assert np.array_equal(r[:9], u0) and not r[9:27].any()
    assert np.array_equal(r[27:], np.ones(2 * 2 * 9))
