"""Relaxed (iteration-dependent) precision of the outer product on the GPU (aao_options.relax_matvec):
the FP32 product against the FP64 oracle within its rigorous rounding bound, and relaxed solves
against the FP64-product solve and the oracle's solution."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.relaxed import gamma
from oracle.solve import OracleOptions, build, solve as oracle_solve

from gpu_util import dev, host, to_dev, torch, zeros

pytestmark = pytest.mark.gpu

G32 = gamma(32)


def make(ns, nt, s, method="radau", kap=None, prec="fp32", relax=0.0, tol=1e-10, T=1.0):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make as tab
    dev()
    return Solver(ns, T, nt, tableau=tab(method, s), kappa=None if kap is None else to_dev(kap), prec_P=prec,
                  inner_maxit=3, inner_tol=1e-3, tol=tol, relax_matvec=relax)


PRODUCT_CASES = [((24, 20), 4, 3, "radau", False), ((7, 6, 5), 3, 2, "gauss", False), ((16, 13), 3, 2, "radau", True),
                 ((6, 5, 7), 2, 3, "radau", True), ((33, 8), 5, 1, "radau", False)]


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("ns,nt,s,method,with_kappa", PRODUCT_CASES)
def test_fp32_product_within_its_rounding_bound(ns, nt, s, method, with_kappa, transpose):
    """|fl32(A x) - A x| <= gamma_32 absy entry by entry (A x from the FP64 oracle), and absy
    bounds |A| |x| of the assembled operator from above (the expression tree's absolute value
    can only add magnitudes), so the bound is at least the textbook one."""
    kap = None
    if with_kappa:
        kap = np.exp(synth.gaussian_random_field(ns, 0.2, 0.5, synth.rng_for(4, "kappa"), with_boundary=True))
    S = make(ns, nt, s, method, kap)
    op = build(ns, 1.0, nt, method, s, kappa=kap)
    for seed in (1, 2):
        x = synth.random_vector(op.n_st, 300 + seed)
        y, absy = S.matvec_relaxed(to_dev(x), zeros(op.n_st), zeros(op.n_st), transpose=transpose)
        y, absy = host(y), host(absy)
        ref = op.rmatvec(x) if transpose else op.matvec(x)
        err = np.abs(y - ref)
        assert np.all(err <= G32 * absy * (1 + 1e-6) + 1e-300), float(np.max(err / (G32 * absy + 1e-300)))
        if op.n_st <= 6000:
            D = sp.csr_matrix(op.dense())
            if transpose:
                D = D.T.tocsr()
            textbook = abs(D) @ np.abs(x)
            assert np.all(absy >= textbook * (1 - 1e-6))
        # the FP32 product is not the FP64 one (the test would pass vacuously otherwise)
        assert np.max(err) > 0.0


def _problem(ns, nt, s, seed=5):
    u0 = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(seed, "u0"))
    f = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(seed, "f"))
    return u0, f


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_relaxed_solve_matches_the_fp64_product_solve(prec):
    """Late outer iterations keep the FP32 product (|g_k| small: a large allowance), early ones
    recompute in FP64; the true residual reaches the tolerance and the solution equals the
    FP64-product solve's and the oracle's to the tolerance's level."""
    ns, nt, s = (48, 40), 16, 3
    u0, f = _problem(ns, nt, s)
    tol = 1e-10
    S0 = make(ns, nt, s, prec=prec, tol=tol)
    x0, i0 = S0.solve(to_dev(f), to_dev(u0), zeros(S0.n_st))
    S1 = make(ns, nt, s, prec=prec, tol=tol, relax=1.0)
    x1, i1 = S1.solve(to_dev(f), to_dev(u0), zeros(S1.n_st))
    op = build(ns, 1.0, nt, "radau", s)
    ref = oracle_solve(op, ns, op.rhs(u0, f), OracleOptions(tol=1e-13)).x
    e0 = np.linalg.norm(host(x0) - ref) / np.linalg.norm(ref)
    e1 = np.linalg.norm(host(x1) - ref) / np.linalg.norm(ref)
    print(f"{prec}: FP64 product its {i0.outer_its} err {e0:.2e}; relaxed its {i1.outer_its} "
          f"({i1.relaxed_matvecs} FP32 products) err {e1:.2e}, rel_res {i1.rel_res:.2e}")
    assert i0.relaxed_matvecs == 0
    assert i1.converged and i1.rel_res <= tol and i1.relaxed_matvecs >= 1
    assert i1.outer_its <= i0.outer_its + 1
    assert e1 <= 1e-8
    # the reported residual is the true FP64 one
    rhs = S1.rhs(to_dev(f), to_dev(u0), zeros(S1.n_st))
    r = rhs - S1.matvec(x1, zeros(S1.n_st))
    assert abs(float(torch.linalg.norm(r) / torch.linalg.norm(rhs)) - i1.rel_res) <= 1e-12


def test_every_product_in_fp32_still_reports_the_true_residual():
    """An allowance so large that every product is kept in FP32: the iteration then stalls near
    FP32 accuracy, and the stopping test (on the true FP64 residual) reports that honestly."""
    ns, nt, s = (32, 28), 8, 2
    u0, f = _problem(ns, nt, s, seed=6)
    S = make(ns, nt, s, relax=1e30, tol=1e-14)
    S.set_tolerances(maxit=12)
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(S.n_st), allow_not_converged=True)
    assert info.relaxed_matvecs == info.outer_its == 12
    rhs = S.rhs(to_dev(f), to_dev(u0), zeros(S.n_st))
    r = rhs - S.matvec(x, zeros(S.n_st))
    true = float(torch.linalg.norm(r) / torch.linalg.norm(rhs))
    assert not info.converged and abs(true - info.rel_res) <= 1e-12 and true > 1e-14


def test_relaxed_adjoint_solve():
    """P_tilde^T and A^T: the transposed FP32 product in the adjoint's outer iteration."""
    ns, nt, s = (40, 36), 8, 3
    tol = 1e-10
    S0 = make(ns, nt, s, tol=tol)
    S1 = make(ns, nt, s, tol=tol, relax=1.0)
    g = to_dev(synth.random_vector(S0.n_st, 77))
    l0, i0 = S0.adjoint_solve(g, zeros(S0.n_st))
    l1, i1 = S1.adjoint_solve(g, zeros(S1.n_st))
    d = float(torch.linalg.norm(l1 - l0) / torch.linalg.norm(l0))
    print(f"adjoint: its {i0.outer_its} / {i1.outer_its}, FP32 products {i1.relaxed_matvecs}, difference {d:.2e}")
    assert i1.converged and i1.relaxed_matvecs >= 1 and d <= 1e-8
