"""Seeded synthetic inputs for the all-at-once Runge--Kutta heat-equation solver.

This module is the only code shared by the CPU oracle and the GPU path.  It
holds no arithmetic of the method (no operator, no preconditioner, no Krylov
step): it only draws the data a user would pass in -- initial data u0, source
f, diffusivity kappa, tracking target -- as float64 numpy arrays laid out
lexicographically with x fastest (index = i + Nx*(j + Ny*k)).

Grid convention (vertex grid, zero Dirichlet data): interior nodes
x_i = i*h, i = 1..N, h = L/(N+1); boundary nodes i = 0 and N+1 are not
unknowns.  Fields that live on all nodes (kappa) have (N+2)^d entries.

Randomness: numpy PCG64, one base seed per workload, sub-seeds by purpose.
Gaussian random fields use the squared-exponential covariance
C(r) = sigma^2 exp(-r^2 / (2 l^2)) sampled exactly through its separable
structure, field = (C1^{1/2} (x) C1^{1/2} [(x) C1^{1/2}]) xi, xi ~ N(0, I).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "Workload", "grid_nodes", "sine_field", "gaussian_random_field",
    "workload_small_2d", "workload_fp32_precond_2d", "workload_lowprec_3d",
    "workload_adjoint_2d", "workload_batched", "random_vector", "rng_for",
]

_PURPOSES = {"u0": 1, "f": 2, "kappa": 3, "target": 4, "noise": 5, "batch": 6,
             "dirs": 7, "vec": 8, "modes": 9}


def rng_for(base_seed: int, purpose: str, index: int = 0) -> np.random.Generator:
    """PCG64 generator for (workload seed, purpose, index)."""
    return np.random.Generator(np.random.PCG64([base_seed, _PURPOSES[purpose], index]))


def grid_nodes(n: int, length: float = 1.0, with_boundary: bool = False) -> np.ndarray:
    """1D node coordinates: interior i*h (i=1..n) or all nodes (i=0..n+1)."""
    h = length / (n + 1)
    idx = np.arange(0, n + 2) if with_boundary else np.arange(1, n + 1)
    return idx * h


def _mesh(ns: Tuple[int, ...], lens: Tuple[float, ...], with_boundary: bool):
    axes = [grid_nodes(n, L, with_boundary) for n, L in zip(ns, lens)]
    # C order with x fastest: array shape (Nz, Ny, Nx) / (Ny, Nx)
    return np.meshgrid(*axes[::-1], indexing="ij")[::-1]


def sine_field(ns, modes, coeffs=None, lens=None) -> np.ndarray:
    """sum_q a_q prod_k sin(m_{q,k} pi x_k / L_k) at interior nodes, flattened."""
    ns = tuple(ns)
    lens = tuple(lens) if lens is not None else (1.0,) * len(ns)
    X = _mesh(ns, lens, False)
    out = np.zeros(X[0].shape)
    if coeffs is None:
        coeffs = [1.0] * len(modes)
    for a, m in zip(coeffs, modes):
        term = np.full(X[0].shape, float(a))
        for k in range(len(ns)):
            term = term * np.sin(m[k] * math.pi * X[k] / lens[k])
        out += term
    return out.reshape(-1).copy()


def _sqrt_cov_1d(x: np.ndarray, ell: float) -> np.ndarray:
    d = x[:, None] - x[None, :]
    C = np.exp(-d * d / (2.0 * ell * ell))
    w, Q = np.linalg.eigh(C)
    w = np.clip(w, 0.0, None)
    return (Q * np.sqrt(w)) @ Q.T


def gaussian_random_field(ns, ell: float, sigma: float, rng: np.random.Generator,
                          lens=None, with_boundary: bool = False) -> np.ndarray:
    """Exact separable squared-exponential GRF sample, flattened (x fastest)."""
    ns = tuple(ns)
    lens = tuple(lens) if lens is not None else (1.0,) * len(ns)
    roots = [_sqrt_cov_1d(grid_nodes(n, L, with_boundary), ell) for n, L in zip(ns, lens)]
    shape = tuple((n + 2 if with_boundary else n) for n in ns[::-1])
    xi = rng.standard_normal(shape)
    # apply C_k^{1/2} along every axis; array axis a corresponds to grid axis d-1-a
    d = len(ns)
    for a in range(d):
        Rk = roots[d - 1 - a]
        xi = np.moveaxis(np.tensordot(Rk, xi, axes=([1], [a])), 0, a)
    return (sigma * xi).reshape(-1).copy()


def random_vector(n: int, seed: int, index: int = 0) -> np.ndarray:
    return rng_for(seed, "vec", index).standard_normal(n)


@dataclass
class Workload:
    """A heat problem on a vertex grid: what the user passes to the solver."""
    name: str
    dim: int
    n: Tuple[int, ...]
    T: float
    nt: int
    method: str            # "radau" or "gauss"
    s: int
    tol: float
    u0: np.ndarray
    f: np.ndarray          # spatial field, constant in time
    kappa: Optional[np.ndarray] = None  # (N+2)^d nodes, or None for kappa == 1
    target: Optional[np.ndarray] = None
    lens: Tuple[float, ...] = (1.0, 1.0, 1.0)
    extra: dict = field(default_factory=dict)

    @property
    def tau(self) -> float:
        return self.T / self.nt

    @property
    def nx(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_st(self) -> int:
        return self.nx * (self.nt + 1 + self.s * self.nt)


def workload_small_2d(seed: int = 0) -> Workload:
    """2D 32x32 interior FD grid, Radau IIA s=2, 16 steps to T=1, tol 1e-10.

    u0 = sin(pi x) sin(pi y); f = sum of 4 sine modes (k, l) in [1,4]^2 with
    N(0,1) coefficients.
    """
    N = 32
    rng = rng_for(seed, "modes")
    coeffs = rng.standard_normal(4)
    modes = [tuple(int(v) for v in rng.integers(1, 5, size=2)) for _ in range(4)]
    u0 = sine_field((N, N), [(1, 1)])
    f = sine_field((N, N), modes, coeffs)
    return Workload("fd2d_n32_radau2_nt16", 2, (N, N), 1.0, 16, "radau", 2, 1e-10,
                    u0, f, extra={"f_modes": modes, "f_coeffs": coeffs.tolist()})


def workload_fp32_precond_2d(seed: int = 1, N: int = 256, nt: int = 128, s: int = 3) -> Workload:
    """2D 256x256 FD grid, Radau IIA s=3, 128 steps to T=1; GRF u0 and f (l=0.1)."""
    u0 = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "u0"))
    f = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "f"))
    return Workload(f"fd2d_n{N}_radau{s}_nt{nt}", 2, (N, N), 1.0, nt, "radau", s, 1e-8, u0, f)


def workload_lowprec_3d(seed: int = 2, N: int = 96, nt: int = 32, method: str = "radau",
                        s: int = 3) -> Workload:
    """3D 96^3 FD grid, T=0.5, 32 steps; u0 = prod sin(pi x_k) + 1e-2 N(0,1); f = 0."""
    u0 = sine_field((N, N, N), [(1, 1, 1)])
    u0 = u0 + 1e-2 * rng_for(seed, "noise").standard_normal(u0.shape[0])
    f = np.zeros_like(u0)
    return Workload(f"fd3d_n{N}_{method}{s}_nt{nt}", 3, (N, N, N), 0.5, nt, method, s, 1e-8, u0, f)


def workload_adjoint_2d(seed: int = 3, N: int = 128, nt: int = 64, s: int = 3) -> Workload:
    """2D 128x128 variable-diffusivity problem for gradients (kappa = exp(g))."""
    g = gaussian_random_field((N, N), 0.15, 0.5, rng_for(seed, "kappa"), with_boundary=True)
    kappa = np.exp(g)
    u0 = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "u0"))
    f = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "f"))
    target = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "target"))
    return Workload(f"fd2d_kappa_n{N}_radau{s}_nt{nt}", 2, (N, N), 1.0, nt, "radau", s, 1e-8,
                    u0, f, kappa=kappa, target=target)


def fd_directions(n: int, count: int, seed: int = 3) -> np.ndarray:
    """Unit-norm N(0, I) directions for finite-difference gradient checks."""
    D = rng_for(seed, "dirs").standard_normal((count, n))
    return D / np.linalg.norm(D, axis=1, keepdims=True)


def workload_batched(seed: int = 4, count: int = 64, sides=(32, 48, 64, 96, 128, 192, 256),
                     steps=(16, 32, 64, 128), stages=(2, 3)) -> List[Workload]:
    """`count` independent 2D problems with seeded uneven (N, n_t, s)."""
    rng = rng_for(seed, "batch")
    out = []
    for p in range(count):
        N = int(rng.choice(sides))
        nt = int(rng.choice(steps))
        s = int(rng.choice(stages))
        u0 = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "u0", p))
        f = gaussian_random_field((N, N), 0.1, 1.0, rng_for(seed, "f", p))
        out.append(Workload(f"batch{p}_n{N}_radau{s}_nt{nt}", 2, (N, N), 1.0, nt, "radau", s,
                            1e-8, u0, f))
    return out
