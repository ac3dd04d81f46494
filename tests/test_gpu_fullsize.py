"""Full-size checks at the configurations the benchmark times.

* 256x256, Radau IIA s=3, 128 steps: the FP64 matvec element by element against the
  oracle (33.6M unknowns), and the FP32-preconditioned solve checked with the
  oracle's own matvec (true residual <= 1e-8) and against the exact all-at-once
  solution (oracle.spectral, mode by mode in the sine basis) to 1e-8.
* 96^3, Gauss s=2 / Radau s=3, 32 steps: matvec on sampled time blocks computed by
  the oracle's operators one block at a time; BF16 / FP16 preconditioned solves
  checked by the oracle's matvec (true residual <= 1e-8) and against the exact
  solution to 1e-8.
"""
import numpy as np
import pytest

import synth
from oracle.solve import build

from gpu_util import dev, host, rel_max, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def _solver(w, prec, **kw):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make
    dev()
    return Solver(w.n, w.T, w.nt, tableau=make(w.method, w.s), prec_P=prec, tol=w.tol, **kw)


def _true_residual(op, x, rhs):
    r = rhs - op.matvec(x)
    return np.linalg.norm(r) / np.linalg.norm(rhs)


def test_fd2d_256_matvec_full_and_fp32_solve():
    w = synth.workload_fp32_precond_2d()
    op = build(w.n, w.T, w.nt, w.method, w.s)
    S = _solver(w, "fp32", inner_maxit=3, inner_tol=1e-3)
    x = synth.random_vector(op.n_st, 3)
    y = host(S.matvec(to_dev(x), zeros(op.n_st)))
    assert rel_max(y, op.matvec(x)) <= 1e-13
    xs, info = S.solve(to_dev(w.f), to_dev(w.u0), zeros(op.n_st))
    xs = host(xs)
    rhs = op.rhs(w.u0, w.f)
    assert info.converged and _true_residual(op, xs, rhs) <= 1e-8
    exact = _exact(w, op, rhs)
    err = np.linalg.norm(xs - exact) / np.linalg.norm(exact)
    print(f"fp32: outer its {info.outer_its}, error vs the exact solution {err:.2e}")
    assert err <= 1e-8


def _exact(w, op, rhs):
    from oracle import spectral
    from oracle.tableau import tableau
    A, b, _ = tableau(w.method, w.s)
    return spectral.solve(w.n, op.tau, w.nt, A, b, rhs)


def _sampled_matvec_blocks(op, x, blocks):
    """Oracle rows of A x for the listed time blocks n (v_{n+1} and V_{n,i})."""
    v, V = op.split(x)
    out = {}
    for n in blocks:
        acc = v[n + 1] - v[n]
        for i in range(op.s):
            acc = acc - op.tau * op.b[i] * V[n, i]
        out[("v", n + 1)] = acc
        for i in range(op.s):
            W = v[n].copy()
            for j in range(op.s):
                W = W + op.tau * op.A[i, j] * V[n, j]
            out[("V", n, i)] = V[n, i] + op.K @ W
    return out


@pytest.mark.parametrize("method,s", [("gauss", 2), ("radau", 3)])
def test_fd3d_96_matvec_sampled(method, s):
    w = synth.workload_lowprec_3d(method=method, s=s)
    op = build(w.n, w.T, w.nt, w.method, w.s)
    S = _solver(w, "fp32")
    x = synth.random_vector(op.n_st, 4)
    y = host(S.matvec(to_dev(x), zeros(op.n_st)))
    yv, yV = op.split(y)
    for key, ref in _sampled_matvec_blocks(op, x, [0, 13, w.nt - 1]).items():
        got = yv[key[1]] if key[0] == "v" else yV[key[1], key[2]]
        assert rel_max(got, ref) <= 1e-13, key


@pytest.mark.parametrize("method,s", [("gauss", 2), ("radau", 3)])
def test_fd3d_96_lowprec_solves_against_exact_solution(method, s):
    w = synth.workload_lowprec_3d(method=method, s=s)
    op = build(w.n, w.T, w.nt, w.method, w.s)
    rhs = op.rhs(w.u0, w.f)
    exact = _exact(w, op, rhs)
    for prec in ("bf16", "fp16"):
        S = _solver(w, prec, inner_maxit=3, inner_tol=1e-3)
        xs, info = S.solve(to_dev(w.f), to_dev(w.u0), zeros(op.n_st))
        xs = host(xs)
        S.close()
        err = np.linalg.norm(xs - exact) / np.linalg.norm(exact)
        print(f"{method}{s} {prec}: outer its {info.outer_its} rel_res {info.rel_res:.2e} "
              f"error vs the exact solution {err:.2e}")
        assert info.converged
        assert _true_residual(op, xs, rhs) <= 1e-8
        assert err <= 1e-8
