"""Pins of the oracle's all-at-once solution: discrete eigenmode closed form and
sequential RK time stepping (Sec. 2)."""
import math
from collections import defaultdict

import numpy as np
import pytest

import synth
from oracle.sequential import sequential_rk
from oracle.solve import OracleOptions, build, solve

# Radau IIA s=2 in closed form and its stability function (Hairer & Wanner).
A2 = np.array([[5 / 12, -1 / 12], [3 / 4, 1 / 4]])


def R_radau2(z):
    return (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)


def closed_form_small_2d(w):
    """Exact discrete solution of the 32x32, s=2, 16-step problem, mode by mode.

    phi_kl = sin(k pi x) sin(l pi y) is an eigenvector of the FD Laplacian K with
    lambda_kl = (4/h^2)(sin^2(k pi h/2) + sin^2(l pi h/2)).  For a mode with
    amplitude y_n and constant forcing amplitude c_f the stage system reads
    (I + tau lambda A) V = (c_f - lambda y_n) e, and with z = -tau lambda
    y_{n+1} = R(z) y_n + tau c_f Q(z), Q(z) = (R(z) - 1)/z.
    """
    N = w.n[0]
    h = 1.0 / (N + 1)
    amp = defaultdict(lambda: [0.0, 0.0])          # mode -> [y0, c_f]
    amp[(1, 1)][0] += 1.0
    for a, m in zip(w.extra["f_coeffs"], w.extra["f_modes"]):
        amp[tuple(m)][1] += a
    nt, tau = w.nt, w.tau
    v = np.zeros((nt + 1, N * N))
    V = np.zeros((nt, 2, N * N))
    for (k, l), (y0, cf) in amp.items():
        lam = 4 / h ** 2 * (math.sin(k * math.pi * h / 2) ** 2 + math.sin(l * math.pi * h / 2) ** 2)
        z = -tau * lam
        R = R_radau2(z)
        Q = (R - 1) / z
        phi = synth.sine_field((N, N), [(k, l)])
        y = y0
        for n in range(nt):
            st = np.linalg.solve(np.eye(2) + tau * lam * A2, (cf - lam * y) * np.ones(2))
            v[n] += y * phi
            V[n, 0] += st[0] * phi
            V[n, 1] += st[1] * phi
            y = R * y + tau * cf * Q
        v[nt] += y * phi
    return np.concatenate([v.ravel(), V.ravel()])


def test_closed_form_eigenmodes_small_2d():
    w = synth.workload_small_2d()
    op = build(w.n, w.T, w.nt, w.method, w.s)
    rhs = op.rhs(w.u0, w.f)
    r = solve(op, w.n, rhs, OracleOptions(tol=1e-13, inner_maxit=5, inner_tol=1e-6))
    assert r.converged
    xc = closed_form_small_2d(w)
    assert np.linalg.norm(r.x - xc) <= 1e-12 * np.linalg.norm(xc)
    # unforced single mode is scaled by exactly R(-tau lambda)^n
    op1 = build(w.n, w.T, w.nt, w.method, w.s)
    rhs1 = op1.rhs(w.u0, np.zeros_like(w.f))
    r1 = solve(op1, w.n, rhs1, OracleOptions(tol=1e-13))
    h = 1.0 / 33
    lam = 8 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    vT = r1.x[w.nt * op1.nx:(w.nt + 1) * op1.nx]
    assert np.allclose(vT, R_radau2(-w.tau * lam) ** w.nt * w.u0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("ns,nt,method,s,T", [((16, 16), 8, "radau", 3, 1.0),
                                               ((8, 8, 8), 4, "gauss", 2, 0.5),
                                               ((12, 10), 6, "radau", 2, 1.0)])
def test_all_at_once_equals_sequential(ns, nt, method, s, T):
    op = build(ns, T, nt, method, s)
    u0 = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(11, "u0"))
    f = synth.gaussian_random_field(ns, 0.2, 1.0, synth.rng_for(11, "f"))
    xs = sequential_rk(op, u0, f)
    r = solve(op, ns, op.rhs(u0, f), OracleOptions(tol=1e-13))
    assert r.converged
    assert np.linalg.norm(r.x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_all_at_once_equals_sequential_kappa():
    ns = (12, 12)
    g = synth.gaussian_random_field(ns, 0.15, 0.5, synth.rng_for(3, "kappa"), with_boundary=True)
    op = build(ns, 1.0, 6, "radau", 3, kappa=np.exp(g))
    u0 = synth.random_vector(op.nx, 1)
    f = synth.random_vector(op.nx, 2)
    xs = sequential_rk(op, u0, f)
    r = solve(op, ns, op.rhs(u0, f), OracleOptions(tol=1e-13))
    assert np.linalg.norm(r.x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_all_at_once_equals_sequential_q1():
    # Q1 finite elements: M is the FE mass matrix in Eq. (update_solution) and in Theta_hat
    ns = (9, 11)
    op = build(ns, 1.0, 5, "radau", 2, disc="q1")
    u0 = synth.random_vector(op.nx, 1)
    f = synth.random_vector(op.nx, 2)
    xs = sequential_rk(op, u0, f)
    r = solve(op, ns, op.rhs(u0, f), OracleOptions(tol=1e-13))
    assert r.converged
    assert np.linalg.norm(r.x - xs) <= 1e-11 * np.linalg.norm(xs)
