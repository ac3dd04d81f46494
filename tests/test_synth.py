"""The seeded input generators (synth/): the Gaussian random fields have exactly the stated
separable squared-exponential covariance, the layout is x fastest, seeding is reproducible, and
the workloads have the stated shapes."""
import math

import numpy as np
import pytest

import synth


class _Basis:
    """Stands in for a generator: standard_normal returns the k-th unit vector."""

    def __init__(self, k):
        self.k = k

    def standard_normal(self, shape):
        e = np.zeros(int(np.prod(shape)))
        e[self.k] = 1.0
        return e.reshape(shape)


def _linear_map(ns, ell, sigma, lens=None, with_boundary=False):
    n = int(np.prod([v + 2 if with_boundary else v for v in ns]))
    cols = [synth.gaussian_random_field(ns, ell, sigma, _Basis(k), lens, with_boundary) for k in range(n)]
    return np.stack(cols, axis=1)


def _cov_1d(n, L, ell, with_boundary):
    x = synth.grid_nodes(n, L, with_boundary)
    return np.exp(-(x[:, None] - x[None, :]) ** 2 / (2 * ell * ell))


@pytest.mark.parametrize("ns,lens,ell,sigma,bnd", [((6, 5), None, 0.3, 1.0, False), ((4, 3, 5), (1.0, 2.0, 0.5), 0.4, 0.5, False),
                                                   ((5, 4), None, 0.15, 0.5, True)])
def test_grf_covariance_is_the_separable_squared_exponential(ns, lens, ell, sigma, bnd):
    """field = L xi with L L^T = sigma^2 (C_z (x) C_y (x) C_x): unit marginal variance for sigma = 1,
    the slowest axis first in the Kronecker product (x fastest in memory)."""
    Lmap = _linear_map(ns, ell, sigma, lens, bnd)
    lens_ = lens or (1.0,) * len(ns)
    C = np.ones((1, 1))
    for a in reversed(range(len(ns))):
        C = np.kron(C, _cov_1d(ns[a], lens_[a], ell, bnd))
    assert np.abs(Lmap @ Lmap.T - sigma ** 2 * C).max() < 1e-10
    assert np.allclose(np.diag(Lmap @ Lmap.T), sigma ** 2)


def test_grf_x_is_the_fastest_axis():
    """Consecutive entries are neighbours along x: with different spacings along x and y, the
    correlation of entries 0 and 1 follows the x spacing and that of entries 0 and n_x the y spacing."""
    ns, ell = (4, 40), 0.2                      # x: 4 points on [0, 1]; y: 40 points on [0, 1]
    Lmap = _linear_map(ns, ell, 1.0)
    C = Lmap @ Lmap.T
    hx, hy = 1 / 5, 1 / 41
    assert abs(C[0, 1] - math.exp(-hx * hx / (2 * ell * ell))) < 1e-10          # (i, j) -> (i + 1, j)
    assert abs(C[0, ns[0]] - math.exp(-hy * hy / (2 * ell * ell))) < 1e-10      # (i, j) -> (i, j + 1)


def test_seeding_is_reproducible_and_separated_by_purpose():
    a = synth.gaussian_random_field((8, 7), 0.1, 1.0, synth.rng_for(1, "u0"))
    b = synth.gaussian_random_field((8, 7), 0.1, 1.0, synth.rng_for(1, "u0"))
    c = synth.gaussian_random_field((8, 7), 0.1, 1.0, synth.rng_for(1, "f"))
    d = synth.gaussian_random_field((8, 7), 0.1, 1.0, synth.rng_for(1, "u0", 1))
    assert np.array_equal(a, b) and not np.allclose(a, c) and not np.allclose(a, d)
    assert np.array_equal(synth.random_vector(10, 3), synth.random_vector(10, 3))


def test_sine_field_is_the_interior_mode():
    f = synth.sine_field((5, 4), [(2, 1)])
    X = synth.grid_nodes(5)
    Y = synth.grid_nodes(4)
    assert np.abs(f - np.outer(np.sin(np.pi * Y), np.sin(2 * np.pi * X)).ravel()).max() < 1e-15


def test_workload_shapes():
    w = synth.workload_small_2d()
    assert (w.n, w.nt, w.s, w.method, w.T, w.tol) == ((32, 32), 16, 2, "radau", 1.0, 1e-10)
    assert np.abs(w.u0 - synth.sine_field((32, 32), [(1, 1)])).max() == 0.0
    w = synth.workload_fp32_precond_2d(N=16, nt=8)                       # the benchmark recipe, small
    assert (w.n, w.nt, w.s, w.T, w.tol) == ((16, 16), 8, 3, 1.0, 1e-8) and w.u0.shape == (256,)
    ws = synth.workload_batched(count=64)
    assert len(ws) == 64 and {x.s for x in ws} <= {2, 3}
    assert {x.n[0] for x in ws} <= {32, 48, 64, 96, 128, 192, 256} and {x.nt for x in ws} <= {16, 32, 64, 128}
