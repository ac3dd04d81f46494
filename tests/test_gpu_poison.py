"""Reads of uninitialised workspace: with AAO_POISON_WORKSPACE set, every device allocation of a
handle starts as 0xFF bytes (NaN in every floating-point type).  A solve and an adjoint solve on a
poisoned handle must equal those on an ordinary handle bit for bit, so no kernel reads workspace
(ghost rows, padding, reduction partials, Krylov bases, staged stencils) before writing it."""
import numpy as np
import pytest

import synth

from gpu_util import dev, to_dev, torch, zeros

pytestmark = pytest.mark.gpu

# (grid, nt, s, P precision, kappa field, discretisation): the cluster V-cycle (2D), the level
# kernels and the batched tail (3D), 16-bit scaled storage, Q1
CASES = [((40, 36), 4, 3, "fp32", False, "fd"), ((34, 37), 3, 2, "fp64", True, "fd"),
         ((14, 12, 10), 2, 2, "fp32", False, "fd"), ((48, 40), 3, 2, "bf16", False, "fd"),
         ((24, 20), 3, 2, "fp32", False, "q1")]


def _solver(ns, nt, s, prec, kappa, disc):
    from paper_2609_16863_gb300 import Solver, radau_iia
    return Solver(ns, 1.0, nt, tableau=radau_iia(s), prec_P=prec, kappa=kappa, disc=disc, tol=1e-9,
                  inner_maxit=3, inner_tol=1e-3)


@pytest.mark.parametrize("ns,nt,s,prec,var,disc", CASES)
def test_poisoned_workspace_gives_identical_results(monkeypatch, ns, nt, s, prec, var, disc):
    dev()
    kap = None
    if var:
        kap = to_dev(np.exp(synth.gaussian_random_field(ns, 0.15, 0.5, synth.rng_for(3, "kappa"),
                                                        with_boundary=True)))
    monkeypatch.delenv("AAO_POISON_WORKSPACE", raising=False)
    plain = _solver(ns, nt, s, prec, kap, disc)
    monkeypatch.setenv("AAO_POISON_WORKSPACE", "1")
    poisoned = _solver(ns, nt, s, prec, kap, disc)
    monkeypatch.delenv("AAO_POISON_WORKSPACE")
    f = to_dev(synth.random_vector(plain.nx, 1))
    u0 = to_dev(synth.random_vector(plain.nx, 2))
    xa, ia = plain.solve(f, u0, zeros(plain.n_st))
    xb, ib = poisoned.solve(f, u0, zeros(plain.n_st))
    torch.cuda.synchronize()
    assert ia.converged and ib.converged and ia.outer_its == ib.outer_its
    assert bool(torch.isfinite(xb).all())
    assert torch.equal(xa, xb)
    g = to_dev(synth.random_vector(plain.n_st, 3))
    la, _ = plain.adjoint_solve(g, zeros(plain.n_st), allow_not_converged=True)
    lb, _ = poisoned.adjoint_solve(g, zeros(plain.n_st), allow_not_converged=True)
    torch.cuda.synchronize()
    assert torch.equal(la, lb)
