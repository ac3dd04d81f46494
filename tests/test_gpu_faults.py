"""Failure paths through the C ABI, injected from the host: every one returns a status and leaves
the context usable (none of them faults, traps or hangs the GPU)."""
import numpy as np
import pytest

import synth
from oracle.solve import OracleOptions, build, solve as oracle_solve

from gpu_util import dev, host, to_dev, torch, zeros

pytestmark = pytest.mark.gpu

NONFINITE, NOT_CONVERGED, BREAKDOWN = -6, -4, -5


def make(ns=(24, 20), nt=4, s=3, prec="fp32", **kw):
    from paper_2609_16863_gb300 import Solver, radau_iia
    dev()
    return Solver(ns, 1.0, nt, tableau=radau_iia(s), prec_P=prec, inner_maxit=3, inner_tol=1e-3, **kw)


def _status(fn):
    from paper_2609_16863_gb300._lib import AaoError
    try:
        fn()
    except AaoError as e:
        return e.status
    return 0


@pytest.mark.parametrize("where", ["f", "u0"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_input_returns_status_and_handle_stays_usable(where, bad):
    S = make()
    f = synth.random_vector(S.nx, 1)
    u0 = synth.random_vector(S.nx, 2)
    g = f.copy() if where == "f" else u0.copy()
    g[S.nx // 3] = bad
    args = (to_dev(g), to_dev(u0)) if where == "f" else (to_dev(f), to_dev(g))
    assert _status(lambda: S.solve(*args, zeros(S.n_st))) == NONFINITE
    # the same handle still solves a clean problem afterwards
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))
    assert info.converged and info.rel_res <= 1e-8


def test_maxit_returns_not_converged_with_the_iterate():
    S = make(maxit=1, tol=1e-12)
    f = synth.random_vector(S.nx, 3)
    u0 = synth.random_vector(S.nx, 4)
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(S.n_st), allow_not_converged=True)
    assert not info.converged and info.outer_its == 1
    rhs = S.rhs(to_dev(f), to_dev(u0), zeros(S.n_st))
    r = rhs - S.matvec(x, zeros(S.n_st))
    rel = float(torch.linalg.norm(r) / torch.linalg.norm(rhs))
    assert 0.0 < rel < 1.0 and abs(rel - info.rel_res) <= 1e-10       # x is the iterate the status reports
    assert _status(lambda: S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))) == NOT_CONVERGED


def test_zero_rhs_returns_zero_without_iterating():
    S = make()
    x, info = S.solve(zeros(S.nx), zeros(S.nx), to_dev(np.ones(S.n_st)))
    assert info.converged and info.outer_its == 0 and float(torch.abs(x).max()) == 0.0


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_storage_survives_values_beyond_fp16_range(prec):
    """A source of size 1e7 (FP16's largest value is 65504): the per-row power-of-two scales keep
    every stored row in range, and the FP64 outer iteration reaches the FP64 solution.  Stored
    without scaling the same right-hand side overflows (tests/test_oracle_lowprec.py)."""
    ns, nt, s = (24, 20), 4, 3
    S = make(ns, nt, s, prec=prec, tol=1e-10)
    u0 = synth.random_vector(S.nx, 5)
    f = 1e7 * synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(5, "f"))
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))
    op = build(ns, 1.0, nt, "radau", s)
    ref = oracle_solve(op, ns, op.rhs(u0, f), OracleOptions(tol=1e-13))
    err = np.linalg.norm(host(x) - ref.x) / np.linalg.norm(ref.x)
    print(f"{prec}: |f| max {np.abs(f).max():.2e}, outer its {info.outer_its}, error vs FP64 oracle {err:.2e}")
    assert info.converged and err <= 1e-8


def test_nonfinite_kappa_is_refused_with_a_status():
    from paper_2609_16863_gb300 import Solver, radau_iia
    dev()
    ns = (16, 12)
    kap = np.ones((ns[0] + 2) * (ns[1] + 2))
    kap[40] = np.nan
    st = _status(lambda: Solver(ns, 1.0, 4, tableau=radau_iia(2), kappa=to_dev(kap), prec_P="fp32"))
    if st == 0:
        S = Solver(ns, 1.0, 4, tableau=radau_iia(2), kappa=to_dev(kap), prec_P="fp32")
        st = _status(lambda: S.solve(to_dev(np.ones(S.nx)), to_dev(np.ones(S.nx)), zeros(S.n_st)))
    assert st in (NONFINITE, BREAKDOWN), st
    # the context stays usable
    S = make()
    _, info = S.solve(to_dev(synth.random_vector(S.nx, 6)), to_dev(synth.random_vector(S.nx, 7)), zeros(S.n_st))
    assert info.converged
