"""GPU adjoint path vs the FP64 oracle and against central finite differences."""
import numpy as np
import pytest

import synth
from oracle.adjoint import adjoint_solve, grad_f, grad_kappa, tracking_dJdx
from oracle.solve import OracleOptions, build, solve as oracle_solve

from gpu_util import dev, host, rel_max, to_dev, torch, zeros

pytestmark = pytest.mark.gpu

KW = dict(inner_maxit=3, inner_tol=1e-6, mg_cycles=3, mg_pre=2, mg_post=2, mg_omega=0.8)


def solver(ns, nt, s, kap, prec="fp64", tol=1e-12, T=0.5):
    from paper_2609_16863_gb300 import Solver, radau_iia
    dev()
    return Solver(ns, T, nt, tableau=radau_iia(s), kappa=None if kap is None else to_dev(kap), prec_P=prec,
                  tol=tol, **KW)


def data(ns, seed=9):
    kap = np.exp(synth.gaussian_random_field(ns, 0.15, 0.5, synth.rng_for(seed, "kappa"), with_boundary=True))
    u0 = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(seed, "u0"))
    f = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(seed, "f"))
    tgt = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(seed, "target"))
    return kap, u0, f, tgt


def test_dot_product_identity():
    ns, nt, s = (20, 18), 4, 3
    kap, *_ = data(ns)
    S = solver(ns, nt, s, kap)
    x = to_dev(synth.random_vector(S.n_st, 1))
    y = to_dev(synth.random_vector(S.n_st, 2))
    Ax = S.matvec(x, zeros(S.n_st))
    ATy = S.matvec(y, zeros(S.n_st), transpose=True)
    a = float(torch.dot(Ax, y))
    b = float(torch.dot(x, ATy))
    assert abs(a - b) <= 1e-13 * abs(a)


@pytest.mark.parametrize("ns,nt,s", [((16, 14), 4, 3), ((8, 7, 9), 3, 2)])
def test_adjoint_solve_and_gradients_match_oracle(ns, nt, s):
    kap, u0, f, tgt = data(ns)
    S = solver(ns, nt, s, kap)
    x = host(S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))[0])
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    g = tracking_dJdx(op, x, tgt)
    lam_d = zeros(S.n_st)
    gf_d = zeros(S.nx)
    nnode = int(np.prod([n + 2 for n in ns]))
    gk_d = zeros(nnode)
    _, info = S.adjoint_solve(to_dev(g), lam_d, x_fwd=to_dev(x), grad_f=gf_d, grad_kappa=gk_d)
    lam = host(lam_d)
    ref, its, rr, ok = adjoint_solve(op, ns, g, tol=1e-12, inner_maxit=3, inner_tol=1e-6, omega=0.8)
    assert info.converged and ok and info.outer_its == its
    assert np.linalg.norm(lam - ref) <= 1e-10 * np.linalg.norm(ref)
    assert rel_max(host(gf_d), grad_f(op, lam)) <= 1e-12
    assert rel_max(host(gk_d), grad_kappa(op, ns, lam, x)) <= 1e-11


def _J(S, f, u0, tgt):
    x = S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))[0]
    xh = host(x)
    lo = S.nt * S.nx
    d = xh[lo: lo + S.nx] - tgt
    return 0.5 * d @ d + 0.5e-4 * f @ f


def test_gradients_against_central_differences():
    """h = 1e-6, forward solves to 1e-13 so solver noise stays far below the 1e-5 target."""
    ns, nt, s = (12, 12), 4, 3
    kap, u0, f, tgt = data(ns, seed=4)
    S = solver(ns, nt, s, kap, tol=1e-13)
    x = host(S.solve(to_dev(f), to_dev(u0), zeros(S.n_st))[0])
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    gf_d = zeros(S.nx)
    gk_d = zeros(kap.size)
    S.adjoint_solve(to_dev(tracking_dJdx(op, x, tgt)), zeros(S.n_st), x_fwd=to_dev(x), grad_f=gf_d,
                    grad_kappa=gk_d)
    gf = host(gf_d) + 1e-4 * f
    gk = host(gk_d)
    h = 1e-6
    # 20 seeded directions each; relative bound with the quotient's noise measured from h to 2h
    for d in synth.fd_directions(f.size, 20, seed=5):
        q = [(_J(S, f + e * d, u0, tgt) - _J(S, f - e * d, u0, tgt)) / (2 * e) for e in (h, 2 * h)]
        assert abs(q[0] - gf @ d) <= 1e-5 * abs(q[0]) + 4 * abs(q[0] - q[1])
    for d in synth.fd_directions(kap.size, 20, seed=6):
        q = []
        for e in (h, 2 * h):
            Sp = solver(ns, nt, s, kap + e * d, tol=1e-13)
            Sm = solver(ns, nt, s, kap - e * d, tol=1e-13)
            q.append((_J(Sp, f, u0, tgt) - _J(Sm, f, u0, tgt)) / (2 * e))
            Sp.close()
            Sm.close()
        assert abs(q[0] - gk @ d) <= 1e-5 * abs(q[0]) + 4 * abs(q[0] - q[1])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_precision_adjoint_gradient(prec):
    ns, nt, s = (24, 24), 4, 3
    kap, u0, f, tgt = data(ns, seed=7)
    S64 = solver(ns, nt, s, kap)
    x = host(S64.solve(to_dev(f), to_dev(u0), zeros(S64.n_st))[0])
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    g = to_dev(tracking_dJdx(op, x, tgt))
    out = {}
    for p, S in (("fp64", S64), (prec, solver(ns, nt, s, kap, prec=prec, tol=1e-12))):
        gk = zeros(kap.size)
        S.adjoint_solve(g, zeros(S.n_st), x_fwd=to_dev(x), grad_kappa=gk)
        out[p] = host(gk)
    err = np.linalg.norm(out[prec] - out["fp64"]) / np.linalg.norm(out["fp64"])
    assert err <= 1e-9, err


def test_autograd_function():
    from paper_2609_16863_gb300.autograd import heat_solve
    from paper_2609_16863_gb300 import radau_iia
    ns, nt, s = (10, 9), 3, 2
    kap, u0, f, tgt = data(ns, seed=11)
    cfg = dict(n=ns, T=0.5, nt=nt, tableau=radau_iia(s), prec_P="fp64", tol=1e-13, **KW)
    fd_ = to_dev(f).requires_grad_(True)
    ud = to_dev(u0).requires_grad_(True)
    kd = to_dev(kap).requires_grad_(True)
    x = heat_solve(fd_, ud, kd, **cfg)
    lo = nt * int(np.prod(ns))
    J = 0.5 * ((x[lo: lo + f.size] - to_dev(tgt)) ** 2).sum() + 0.5e-4 * (fd_ ** 2).sum()
    J.backward()
    op = build(ns, 0.5, nt, "radau", s, kappa=kap)
    xr = np.linalg.solve(op.dense(), op.rhs(u0, f))
    lam = np.linalg.solve(op.dense().T, tracking_dJdx(op, xr, tgt))
    assert rel_max(host(fd_.grad), grad_f(op, lam) + 1e-4 * f) <= 1e-9
    assert rel_max(host(ud.grad), lam[: f.size]) <= 1e-9
    assert rel_max(host(kd.grad), grad_kappa(op, ns, lam, xr)) <= 1e-9


def test_checkpointed_gradient_equals_full_storage():
    """Forward states kept every 8 steps and recomputed window by window give the
    same kappa gradient as keeping the whole trajectory (<= 1e-10)."""
    from paper_2609_16863_gb300.autograd import heat_solve
    from paper_2609_16863_gb300 import radau_iia
    ns, nt, s = (20, 18), 20, 3
    kap, u0, f, tgt = data(ns, seed=13)
    grads = []
    for k in (0, 8):
        cfg = dict(n=ns, T=1.0, nt=nt, tableau=radau_iia(s), prec_P="fp64", tol=1e-13, ckpt_every=k, **KW)
        fd_ = to_dev(f).requires_grad_(True)
        kd = to_dev(kap).requires_grad_(True)
        x = heat_solve(fd_, to_dev(u0), kd, **cfg)
        lo = nt * int(np.prod(ns))
        J = 0.5 * ((x[lo: lo + f.size] - to_dev(tgt)) ** 2).sum()
        J.backward()
        grads.append((host(fd_.grad), host(kd.grad)))
    assert rel_max(grads[1][0], grads[0][0]) <= 1e-12
    assert np.linalg.norm(grads[1][1] - grads[0][1]) <= 1e-10 * np.linalg.norm(grads[0][1])


def test_gradients_fd_check_128_checkpointed():
    """128x128, Radau IIA s=3, 64 steps, kappa = exp(GRF): the checkpointed (every 8 steps)
    kappa and f gradients of J = 1/2||u(T)-u_target||^2 + 1/2 1e-4 ||f||^2 against central
    differences (h = 1e-6) on 20 seeded unit directions each.  With h_x = 1/129 and kappa up to
    about e^1.5 the stage block e (x) K has norm ~6e5, so FP64 residuals stall near 1e-11: the
    gradient solves use tol 1e-9 and the reference solves run FGMRES to stagnation.  J is about
    9e3 while the directional derivatives are about 1e-3, so J(+) - J(-) is formed from the state
    difference, 1/2 (d+ - d-).(d+ + d-) with d = u(T) - u_target, instead of subtracting two
    rounded J values; the noise of the quotient is measured as its change from h to 2h, and the
    bound is relative: |fd - g.d| <= 1e-5 |fd| + 4 noise."""
    from paper_2609_16863_gb300.autograd import heat_solve
    from paper_2609_16863_gb300 import Solver, radau_iia
    w = synth.workload_adjoint_2d()
    cfg = dict(n=w.n, T=w.T, nt=w.nt, tableau=radau_iia(w.s), prec_P="fp32", tol=1e-9, maxit=200, ckpt_every=8,
               inner_maxit=3, inner_tol=1e-3)
    lo = w.nt * w.nx

    def solver_for(kap):
        return Solver(w.n, w.T, w.nt, tableau=radau_iia(w.s), kappa=to_dev(kap), prec_P="fp32", inner_maxit=3,
                      inner_tol=1e-3, tol=1e-15, maxit=24)

    def state(S, f):
        x, info = S.solve(to_dev(f), to_dev(w.u0), zeros(S.n_st), allow_not_converged=True)
        assert info.rel_res <= 1e-10, info.rel_res
        return host(x)[lo: lo + w.nx] - w.target

    def quotient(dp, dm, fp, fm, h):
        return (0.5 * (dp - dm) @ (dp + dm) + 0.5e-4 * (fp - fm) @ (fp + fm)) / (2 * h)

    fd_ = to_dev(w.f).requires_grad_(True)
    kd = to_dev(w.kappa).requires_grad_(True)
    x = heat_solve(fd_, to_dev(w.u0), kd, **cfg)
    J = 0.5 * ((x[lo: lo + w.nx] - to_dev(w.target)) ** 2).sum() + 0.5e-4 * (fd_ ** 2).sum()
    J.backward()
    gf, gk = host(fd_.grad), host(kd.grad)
    h = 1e-6
    worst = 0.0
    S0 = solver_for(w.kappa)
    for n, d in enumerate(synth.fd_directions(w.nx, 20, seed=21)):
        q = [quotient(state(S0, w.f + e * d), state(S0, w.f - e * d), w.f + e * d, w.f - e * d, e) for e in (h, 2 * h)]
        err, noise = abs(q[0] - gf @ d), abs(q[0] - q[1])
        print(f"f dir {n}: |fd| {abs(q[0]):.4e} |fd - g.d| {err:.2e} noise {noise:.2e}")
        worst = max(worst, err / (1e-5 * abs(q[0]) + 4 * noise))
        assert err <= 1e-5 * abs(q[0]) + 4 * noise
    S0.close()
    for n, d in enumerate(synth.fd_directions(w.kappa.size, 20, seed=22)):
        q = []
        for e in (h, 2 * h):
            Sp, Sm = solver_for(w.kappa + e * d), solver_for(w.kappa - e * d)
            q.append(quotient(state(Sp, w.f), state(Sm, w.f), w.f, w.f, e))
            Sp.close()
            Sm.close()
        err, noise = abs(q[0] - gk @ d), abs(q[0] - q[1])
        print(f"kappa dir {n}: |fd| {abs(q[0]):.4e} |fd - g.d| {err:.2e} noise {noise:.2e}")
        worst = max(worst, err / (1e-5 * abs(q[0]) + 4 * noise))
        assert err <= 1e-5 * abs(q[0]) + 4 * noise
    print(f"worst error / bound {worst:.2f}")
