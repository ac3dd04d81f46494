"""Pins of the oracle's adjoint solve and gradients: central finite differences of the
tracking functional with dense LU forward solves, and a dense transposed solve."""
import numpy as np
import pytest

import synth
from oracle.adjoint import (adjoint_solve, grad_f, grad_kappa, grad_u0, tracking_dJdx,
                            tracking_J)
from oracle.solve import build


def _setup(ns, nt, s, seed=0):
    rng = np.random.default_rng(seed)
    nnode = int(np.prod([n + 2 for n in ns]))
    kap = np.exp(0.5 * rng.standard_normal(nnode))
    nx = int(np.prod(ns))
    return kap, rng.standard_normal(nx), rng.standard_normal(nx), rng.standard_normal(nx)


def _J(ns, nt, s, kap, f, u0, tgt):
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    x = np.linalg.solve(op.dense(), op.rhs(u0, f))
    return tracking_J(op, x, f, tgt), op, x


@pytest.mark.parametrize("ns,nt,s", [((4, 3), 2, 2), ((3, 3, 2), 2, 3)])
def test_gradients_match_central_differences(ns, nt, s):
    kap, f, u0, tgt = _setup(ns, nt, s)
    J0, op, x = _J(ns, nt, s, kap, f, u0, tgt)
    lam = np.linalg.solve(op.dense().T, tracking_dJdx(op, x, tgt))
    gf = grad_f(op, lam) + 1e-4 * f
    gu = grad_u0(op, lam)
    gk = grad_kappa(op, ns, lam, x)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(f.shape); d /= np.linalg.norm(d)
        fd = (_J(ns, nt, s, kap, f + h * d, u0, tgt)[0] - _J(ns, nt, s, kap, f - h * d, u0, tgt)[0]) / (2 * h)
        assert abs(fd - gf @ d) <= 1e-6 * max(1.0, abs(fd))
        fd = (_J(ns, nt, s, kap, f, u0 + h * d, tgt)[0] - _J(ns, nt, s, kap, f, u0 - h * d, tgt)[0]) / (2 * h)
        assert abs(fd - gu @ d) <= 1e-6 * max(1.0, abs(fd))
        dk = rng.standard_normal(kap.shape); dk /= np.linalg.norm(dk)
        fd = (_J(ns, nt, s, kap + h * dk, f, u0, tgt)[0] - _J(ns, nt, s, kap - h * dk, f, u0, tgt)[0]) / (2 * h)
        assert abs(fd - gk @ dk) <= 1e-6 * max(1.0, abs(fd))


def test_adjoint_fgmres_matches_dense_transpose_solve():
    ns, nt, s = (6, 5), 3, 3
    kap, f, u0, tgt = _setup(ns, nt, s, seed=3)
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    x = np.linalg.solve(op.dense(), op.rhs(u0, f))
    g = tracking_dJdx(op, x, tgt)
    lam, its, rr, ok = adjoint_solve(op, ns, g, tol=1e-13, inner_maxit=5, inner_tol=1e-6, omega=0.8)
    ref = np.linalg.solve(op.dense().T, g)
    assert ok and np.linalg.norm(lam - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("disc,ns,nt,s", [("fd", (5, 4), 3, 3), ("fd", (3, 3, 2), 2, 2), ("q1", (4, 5), 3, 2)])
def test_sequential_adjoint_matches_dense_transpose(disc, ns, nt, s):
    from oracle.sequential import sequential_adjoint_rk
    kap = _setup(ns, nt, s, seed=5)[0] if disc == "fd" else None
    op = build(ns, 0.5, nt, "radau", s, disc=disc, kappa=kap)
    g = synth.random_vector(op.n_st, 9)
    ref = np.linalg.solve(op.dense().T, g)
    assert np.linalg.norm(sequential_adjoint_rk(op, g) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_adjoint_fgmres_matches_backward_adjoint_rk_at_scale():
    """Beyond dense sizes: 40 x 36 with a kappa field, Radau IIA s = 3, 16 steps."""
    from oracle.sequential import sequential_adjoint_rk
    ns, nt, s = (40, 36), 16, 3
    kap = np.exp(synth.gaussian_random_field(ns, 0.15, 0.5, synth.rng_for(3, "kappa"), with_boundary=True))
    op = build(ns, 1.0, nt, "radau", s, kappa=kap)
    g = synth.random_vector(op.n_st, 11)
    lam, its, rr, ok = adjoint_solve(op, ns, g, tol=1e-12, inner_maxit=5, inner_tol=1e-6, omega=0.8)
    ref = sequential_adjoint_rk(op, g)
    assert ok and np.linalg.norm(lam - ref) <= 1e-10 * np.linalg.norm(ref)
