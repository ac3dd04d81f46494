"""Full-size checks at the configuration the benchmark times.

* 256x256, Radau IIA s=3, 128 steps: the FP64 matvec element by element against the
  oracle (33.6M unknowns), and the FP32-preconditioned solve checked with the
  oracle's own matvec (true residual <= 1e-8) and against the FP64-preconditioned
  GPU solve.
* 96^3, Gauss s=2 / Radau s=3, 32 steps: matvec on sampled time blocks computed by
  the oracle's operators one block at a time; BF16 / FP16 preconditioned solves
  checked by the oracle's matvec (true residual <= 1e-8).
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
    S64 = _solver(w, "fp64")
    x64, i64 = S64.solve(to_dev(w.f), to_dev(w.u0), zeros(op.n_st))
    err = np.linalg.norm(xs - host(x64)) / np.linalg.norm(host(x64))
    print(f"fp32 its {info.outer_its} fp64 its {i64.outer_its} rel diff {err:.2e}")
    assert err <= 1e-7


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


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_fd3d_96_lowprec_solve_residual(prec):
    w = synth.workload_lowprec_3d(method="radau", s=3)
    op = build(w.n, w.T, w.nt, w.method, w.s)
    S = _solver(w, prec, inner_maxit=3, inner_tol=1e-3)
    xs, info = S.solve(to_dev(w.f), to_dev(w.u0), zeros(op.n_st))
    print(f"{prec}: outer its {info.outer_its} rel_res {info.rel_res:.2e}")
    assert info.converged
    assert _true_residual(op, host(xs), op.rhs(w.u0, w.f)) <= 1e-8
