"""Low-precision P_tilde on the GPU against the oracle's storage emulation (oracle.lowprec).

The emulation rounds what P_tilde stores to FP32, BF16 or FP16 with the same per-row power-of-two
scales and computes in float32 (Sec. 4-5; the paper's chop simulation of Sec. 5.1), following the
CUDA path's memory plan (gpu_util.gpu_plan).  Given the same stored inputs, a step of the CUDA path
and of the emulation then differ only by float32 rounding order, which moves a stored 16-bit value
by one unit in the last place where the float32 values straddle a rounding boundary.  So:

* one step with identical inputs (a shifted solve; one stage of Rana's sweep built from the GPU's
  own earlier stages) agrees entry by entry within one unit in the last place of the storage format
  plus a float32 noise floor of 2^-18 of the row maximum (entries near zero) where only the step's
  result is stored (a 2D item on a thread-block cluster); where the V-cycles store intermediate
  vectors (3D items), a flip in an intermediate reaches a few neighbouring entries of the result,
  which may then differ by up to 16 units (measured: 9); either way at most 5% of the entries
  differ at all;
* composite results (inner GMRES, P_tilde) pass such flips through tau K, which amplifies them, and
  are compared in the 2-norm against bounds set from measured runs with a margin (BF16 rounding
  flips move inner GMRES's result by up to ~9e-4, P_tilde's by up to ~9e-3);
* FP32 storage rounds nothing the arithmetic has not rounded already; there the two sides differ by
  float32 rounding order alone, amplified on anisotropic grids (up to ~3e-5).
A scale, rounding or memory-plan mistake moves most entries by about a unit (a plan mistake alone:
2-norm ~6e-4 in BF16 for three V-cycles), which the entrywise checks reject.
"""
import numpy as np
import pytest

import synth
from oracle import lowprec as lp
from oracle.precond import Preconditioner
from oracle.solve import build

from gpu_util import dev, gpu_plan, host, lowprec_errors, storage_ulps, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def make(ns, nt, s, precP, precI=None, method="radau", inner_tol=0.0):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make as tab
    dev()
    precI = precI or precP
    S = Solver(ns, 1.0, nt, tableau=tab(method, s), prec_P=precP, prec_Pint=precI, inner_maxit=3,
               inner_tol=inner_tol, mg_cycles=3, mg_pre=2, mg_post=2, mg_omega=0.8)
    op = build(ns, 1.0, nt, method, s)
    P = Preconditioner(op, ns, 3, inner_tol, 3, 2, 2, 0.8)
    return S, op, P


def emulation(P, precP, precI, B, cluster):
    sizes = P.mg[0].sizes
    return lp.StoredPreconditioner(P, precP, precI, gpu_plan(sizes, B, cluster, precI),
                                   gpu_plan(sizes, 1, cluster, precI))


def check_step(what, got, ref, n0, fmt, max_ulps):
    """One step with identical stored inputs: entrywise within max_ulps units in the last place
    (16-bit) or within float32 rounding-order differences (FP32)."""
    e2, emax, _ = lowprec_errors(got, ref)
    if fmt == "fp32":
        print(f"{what} [fp32]: rel2 {e2:.2e} relmax {emax:.2e}")
        assert e2 <= 5e-5, (what, e2)
        return
    ulps, frac = storage_ulps(got, ref, n0, fmt)
    print(f"{what} [{fmt}]: max {ulps:.2f} ulp, {100 * frac:.2f}% of entries differ, rel2 {e2:.2e}")
    assert ulps <= max_ulps, (what, ulps)
    assert frac <= 0.05, (what, frac)


# (grid, fmt, a single 2D item runs on a thread-block cluster, allowed units in the last place)
SHIFTED = [((48, 40), "bf16", True, 1), ((48, 40), "fp16", True, 1), ((48, 40), "fp32", True, 0),
           ((97, 33), "bf16", True, 1), ((64, 64), "fp16", True, 1), ((20, 18, 22), "bf16", False, 16),
           ((16, 16, 16), "fp16", False, 16), ((130, 70), "fp32", True, 0), ((24, 16, 20), "bf16", False, 16)]


@pytest.mark.parametrize("ns,fmt,cluster,ulps", SHIFTED)
def test_shifted_solve_matches_storage_emulation(ns, fmt, cluster, ulps):
    S, op, P = make(ns, 2, 2, fmt)
    E = emulation(P, fmt, fmt, 2, cluster)
    for i in range(2):
        b = synth.random_vector(op.nx, 120 + i)
        x = host(S.shifted_solve(i, to_dev(b), zeros(op.nx)))
        ref = E.mg[i].solve(lp.store_rows(b, ns[0], fmt), 3, E.plan_single).astype(np.float64)
        check_step(f"shifted {ns} stage {i}", x, ref, ns[0], fmt, ulps)


@pytest.mark.parametrize("ns,precP,precI,cluster,ulps", [((48, 40), "bf16", "bf16", True, 4),
                                                         ((48, 40), "fp32", "bf16", True, 4),
                                                         ((64, 64), "fp16", "fp16", True, 4),
                                                         ((12, 10, 14), "fp16", "fp16", False, 16),
                                                         ((33, 17), "fp32", "fp32", True, 0)])
def test_pint_stages_match_storage_emulation(ns, precP, precI, cluster, ulps):
    """Rana's sweep stage by stage: stage i of the emulation is built from the GPU's own stages
    j < i (forward) or j > i (backward), so every stage is one step with nearly identical inputs:
    the right-hand side V_i - tau (LD)_ij K Z_j is itself a float32 result rounded to storage,
    where the two sides may differ by one unit, which the shifted solve spreads over a few
    neighbouring entries (up to 4 units measured on 2D grids, 16 allowed in 3D)."""
    s = 3
    S, op, P = make(ns, 2, s, precP, precI)
    E = emulation(P, precP, precI, 2, cluster)
    nx, dt = op.nx, E.dt
    r = synth.random_vector(s * nx, 130)
    V = E.stP(r.astype(dt)).reshape(s, nx)
    tau = dt(op.tau)
    for tr in (False, True):
        y = host(S.pint_apply(to_dev(r), zeros(s * nx), transpose=tr)).reshape(s, nx)
        for i in range(s):
            acc = V[i].copy()
            for j in range(s):
                cf = P.LD[j, i] if tr else P.LD[i, j]
                if (j > i if tr else j < i) and cf != 0.0:
                    acc = acc - (tau * dt(cf)) * (E.K @ y[j].astype(dt))
            ref = E.shifted_solve(i, E.stI(acc), E.plan_single).astype(np.float64)
            check_step(f"pint {ns} T={tr} stage {i}", y[i], ref, ns[0], precI, ulps)
        # the whole sweep against the emulation's own sweep: flips amplified by tau K
        e2 = lowprec_errors(y.reshape(-1), E.pint(V.reshape(-1), E.plan_single, transpose=tr))[0]
        print(f"pint {ns} T={tr} whole sweep: rel2 {e2:.2e}")
        assert e2 <= {"fp32": 5e-5, "fp16": 1e-3, "bf16": 5e-3}[precI]


INNER_BOUND = {"fp32": 2e-5, "fp16": 1e-3, "bf16": 2e-3}


@pytest.mark.parametrize("ns,nb,precP,precI,cluster", [((48, 40), 4, "bf16", "bf16", True),
                                                       ((128, 128), 4, "fp16", "fp16", True),
                                                       ((20, 18, 22), 3, "bf16", "bf16", False),
                                                       ((64, 64), 3, "fp32", "bf16", True),
                                                       ((40, 36), 5, "fp32", "fp32", True),
                                                       ((48, 40), 40, "bf16", "bf16", False),
                                                       ((64, 32), 36, "fp16", "fp16", False),
                                                       ((16, 16, 24), 4, "bf16", "bf16", False),
                                                       ((64, 64), 12, "bf16", "bf16", True),
                                                       ((256, 256), 16, "fp32", "fp32", True),
                                                       ((256, 256), 12, "bf16", "bf16", True)])
def test_inner_solve_matches_storage_emulation(ns, nb, precP, precI, cluster):
    """Batched inner GMRES (3 fixed iterations) per time block; batches of more than 32 items take
    the level kernels and the on-chip tail instead of one cluster per item, batches of 8 to 32 the
    8-CTA cluster plan (at 256^2 the lean one: level-1 stencil and coarsest inverse read from L2 --
    in BF16 storage converted with their scales by the vector steps -- and a scalar level-0 Jacobi
    weight), which gives the same values as the staged layout."""
    s = 2
    S, op, P = make(ns, nb, s, precP, precI)
    E = emulation(P, precP, precI, nb, cluster)
    R = synth.random_vector(nb * s * op.nx, 140).reshape(nb, s * op.nx)
    Z = host(S.inner_solve(nb, to_dev(R.reshape(-1)), zeros(nb * s * op.nx))[0]).reshape(nb, -1)
    worst = 0.0
    for n in range(min(nb, 5 if op.nx <= 20000 else 2)):
        e2 = lowprec_errors(Z[n], E.inner_solve(R[n], E.plan_batch))[0]
        worst = max(worst, e2)
    print(f"inner {ns} x{nb} [{precP}/{precI}]: worst rel2 {worst:.2e}")
    assert worst <= INNER_BOUND[precI]


@pytest.mark.parametrize("ns,nt,s,precP,precI,cluster", [((32, 32), 4, 3, "bf16", "bf16", True),
                                                         ((32, 32), 4, 3, "fp16", "fp16", True),
                                                         ((32, 32), 4, 3, "fp32", "fp32", True),
                                                         ((32, 32), 4, 3, "fp32", "bf16", True),
                                                         ((10, 9, 8), 3, 2, "bf16", "bf16", False)])
def test_precond_matches_storage_emulation(ns, nt, s, precP, precI, cluster):
    S, op, P = make(ns, nt, s, precP, precI)
    E = emulation(P, precP, precI, nt, cluster)
    r = synth.random_vector(op.n_st, 150)
    bound = {"fp32": 2e-5, "fp16": 1e-2, "bf16": 3e-2}[precI]
    for tr in (False, True):
        z = host(S.precond_apply(to_dev(r), zeros(op.n_st), transpose=tr))
        ref = E.apply_T(r) if tr else E.apply(r)
        e2 = lowprec_errors(z, ref)[0]
        print(f"precond {ns} T={tr} [{precP}/{precI}]: rel2 {e2:.2e}")
        assert e2 <= bound
