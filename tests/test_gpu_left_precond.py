"""Left preconditioning on the GPU (Algorithm 1 with P_L = P_tilde, P_R = I; the paper's parallel
runs, Sec. 5.2) against the oracle's Algorithm 1 (oracle.fgmres.fgmres_split)."""
import numpy as np
import pytest

import synth
from oracle.fgmres import fgmres_split
from oracle.precond import Preconditioner
from oracle.solve import build

from gpu_util import dev, host, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def make(ns, nt, s, prec="fp64", tol=1e-10, mgrit_m=0, method="radau"):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make as tab
    dev()
    itol = 1e-6 if prec == "fp64" else 1e-3
    S = Solver(ns, 1.0, nt, tableau=tab(method, s), prec_P=prec, inner_maxit=3, inner_tol=itol, mg_cycles=3,
               mg_pre=2, mg_post=2, mg_omega=0.8, tol=tol, mgrit_m=mgrit_m, precond_side="left")
    op = build(ns, 1.0, nt, method, s)
    kw = dict(schur="mgrit", mgrit_m=mgrit_m, mgrit_iters=1, mgrit_relax="F") if mgrit_m else {}
    P = Preconditioner(op, ns, 3, itol, 3, 2, 2, 0.8, **kw)
    return S, op, P


@pytest.mark.parametrize("ns,nt,s,m,method", [((24, 20), 4, 3, 0, "radau"), ((32, 32), 8, 2, 4, "radau"),
                                              ((7, 6, 5), 3, 2, 0, "gauss")])
def test_left_preconditioned_solve_matches_oracle(ns, nt, s, m, method):
    S, op, P = make(ns, nt, s, mgrit_m=m, method=method)
    u0 = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(3, "u0"))
    f = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(3, "f"))
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(op.n_st))
    xr, its, rr, ok = fgmres_split(op.matvec, P.apply, lambda v: v.copy(), op.rhs(u0, f), tol=1e-10, restart=20,
                                   maxit=100)
    print(f"left {ns}: GPU its {info.outer_its} oracle its {its}, true residuals {info.rel_res:.2e} / {rr:.2e}")
    assert info.converged and ok and info.outer_its == its
    assert np.linalg.norm(host(x) - xr) <= 1e-10 * np.linalg.norm(xr)
    assert abs(info.rel_res - rr) <= 0.1 * rr + 1e-14        # true residuals agree (rounding level near 1e-13)


def test_left_preconditioned_fp32_against_exact_solution():
    """With P_L applied in FP32 the left-preconditioned residual P^{-1} b - P^{-1} A x carries the
    FP32 rounding of both applies, so it cannot fall far below FP32's unit roundoff (Algorithm 1's
    accuracy depends on u_{P_L}, Sec. 4): the solve runs to 1e-6, and the true residual and the
    error against the exact solution are reported and bounded."""
    from oracle import spectral
    from oracle.tableau import tableau
    ns, nt, s = (48, 48), 16, 3
    S, op, _ = make(ns, nt, s, prec="fp32", tol=1e-6, mgrit_m=4)
    u0 = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(4, "u0"))
    f = synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(4, "f"))
    x, info = S.solve(to_dev(f), to_dev(u0), zeros(op.n_st))
    A, b, _ = tableau("radau", s)
    exact = spectral.solve(ns, op.tau, nt, A, b, op.rhs(u0, f))
    err = np.linalg.norm(host(x) - exact) / np.linalg.norm(exact)
    print(f"left FP32: outer its {info.outer_its}, true residual {info.rel_res:.2e}, error {err:.2e}")
    assert info.converged and info.rel_res <= 1e-5 and err <= 1e-5
