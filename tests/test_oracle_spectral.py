"""Pins of the oracle's exact mode-by-mode solve (oracle.spectral) for constant-coefficient FD."""
import numpy as np
import pytest

import synth
from oracle import spectral
from oracle.sequential import sequential_solve
from oracle.solve import build
from oracle.tableau import tableau


@pytest.mark.parametrize("ns,method,s,nt", [((7, 5), "radau", 2, 4), ((9, 8), "radau", 3, 5),
                                            ((6, 5, 4), "gauss", 2, 3), ((4, 5, 6), "radau", 3, 2)])
def test_spectral_equals_sequential_direct_solve(ns, method, s, nt):
    op = build(ns, 0.7, nt, method, s)
    rhs = synth.random_vector(op.n_st, 17)
    A, b, _ = tableau(method, s)
    x_lu = sequential_solve(op, rhs)
    x_sp = spectral.solve(ns, op.tau, nt, A, b, rhs)
    assert np.abs(x_sp - x_lu).max() <= 1e-13 * np.abs(x_lu).max()


@pytest.mark.parametrize("ns,lens", [((6, 9), None), ((5, 4, 3), None), ((7, 6), (2.0, 0.5))])
def test_eigenvalues_and_transform_diagonalise_K(ns, lens):
    from oracle.operators import operators
    _, K = operators(ns, lens)
    lam = spectral.eigenvalues(ns, lens)
    ev = np.linalg.eigvalsh(K.toarray())
    assert np.abs(np.sort(lam) - ev).max() <= 1e-12 * ev.max()
    # S K S = diag(lambda) with the transform applied column by column
    nx = K.shape[0]
    I = np.eye(nx)
    S = np.stack([spectral.sine(I[:, j], ns) for j in range(nx)], axis=1)
    assert np.abs(S @ S - I).max() <= 1e-13
    assert np.abs(S @ K.toarray() @ S - np.diag(lam)).max() <= 1e-10 * lam.max()


def test_unforced_eigenmode_propagates_by_stability_function():
    # Radau IIA s = 2: R(z) = (1 + z/3) / (1 - 2z/3 + z^2/6) (Hairer--Wanner)
    ns, nt, T = (15, 11), 6, 0.3
    op = build(ns, T, nt, "radau", 2)
    A, b, _ = tableau("radau", 2)
    u0 = synth.sine_field(ns, [(2, 3)])
    h = [1.0 / (n + 1) for n in ns]
    lam = sum(4 / hh ** 2 * np.sin(k * np.pi * hh / 2) ** 2 for hh, k in zip(h, (2, 3)))
    z = -op.tau * lam
    R = (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)
    x = spectral.solve(ns, op.tau, nt, A, b, op.rhs(u0, np.zeros(op.nx)))
    v, _ = op.split(x)
    for n in range(nt + 1):
        assert np.abs(v[n] - R ** n * u0).max() <= 1e-13
