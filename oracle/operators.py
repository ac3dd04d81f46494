"""Spatial operators: stiffness K and mass M on a vertex grid with Dirichlet data.

Test infrastructure only (see the package header).

Sec. 2: after the RK step, space is discretised; K is the stiffness and M the
mass matrix (Eq. discretized_system_stages).  Two discretisations:

* finite differences (FD): M = I, K = -Delta_h, the 5-point (2D) / 7-point
  (3D) Laplacian, or its flux form div(kappa grad u) with nodal kappa averaged
  onto faces, kappa_f = (kappa_P + kappa_nb)/2:
      (K u)_P = sum_axes sum_{+-} kappa_f (u_P - u_{P+-e}) / h_a^2,
  u = 0 on boundary nodes.  kappa == 1 gives the standard Laplacian.
* Q1 finite elements on a tensor mesh: the 1D linear-element matrices
  M1 = h/6 tridiag(1, 4, 1), K1 = 1/h tridiag(-1, 2, -1) restricted to the
  interior nodes, and M = (x)_a M1_a, K = sum_a (x)_{b != a} M1_b (x) K1_a.
* Q2 finite elements (Sec. 5: the paper's second element family) on the same
  tensor construction with 1D quadratic elements (vertex and midpoint nodes).

Layout: lexicographic with x fastest; Kronecker products therefore list the
slowest axis first (kron(Ay, Ax) in 2D).

Pins (tests): K with kappa == 1 against the Kronecker sum of 1D second
differences; the flux form by symmetry, constant-kappa scaling and its energy
u^T K u summed face by face;
Q1 mass row sums and the Jacobi interval of D^{-1} M; the sine eigenpairs of K
through the closed-form solution.
"""
from __future__ import annotations

from functools import reduce

import numpy as np
import scipy.sparse as sp


def _tridiag(n: int, lo: float, d: float, up: float) -> sp.csr_matrix:
    return sp.diags([np.full(n - 1, lo), np.full(n, d), np.full(n - 1, up)], [-1, 0, 1],
                    shape=(n, n), format="csr")


def spacing(ns, lens=None):
    lens = lens if lens is not None else (1.0,) * len(ns)
    return [L / (n + 1) for n, L in zip(ns, lens)]


def stiffness_fd(ns, lens=None, kappa=None) -> sp.csr_matrix:
    """K = -div(kappa grad) by the flux form above; kappa on all (N+2)^d nodes."""
    ns = tuple(int(n) for n in ns)
    d = len(ns)
    hs = spacing(ns, lens)
    shape_i = ns[::-1]                        # interior array shape, x last
    nx = int(np.prod(ns))
    idx = np.arange(nx).reshape(shape_i)
    if kappa is None:
        kap = np.ones(tuple(n + 2 for n in ns[::-1]))
    else:
        kap = np.asarray(kappa, dtype=np.float64).reshape(tuple(n + 2 for n in ns[::-1]))
    interior = tuple(slice(1, n + 1) for n in ns[::-1])
    kP = kap[interior]
    rows, cols, vals = [], [], []
    diag = np.zeros(shape_i)
    for a in range(d):                        # grid axis a -> array axis d-1-a
        ax = d - 1 - a
        for sgn in (-1, 1):
            sl = list(interior)
            sl[ax] = slice(1 + sgn, ns[a] + 1 + sgn)
            kN = kap[tuple(sl)]
            kf = 0.5 * (kP + kN) / (hs[a] * hs[a])
            diag += kf
            # neighbour inside the interior?
            src = [slice(None)] * d
            dst = [slice(None)] * d
            if sgn == 1:
                src[ax] = slice(0, ns[a] - 1)
                dst[ax] = slice(1, ns[a])
            else:
                src[ax] = slice(1, ns[a])
                dst[ax] = slice(0, ns[a] - 1)
            rows.append(idx[tuple(src)].ravel())
            cols.append(idx[tuple(dst)].ravel())
            vals.append(-kf[tuple(src)].ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx, nx)).tocsr()
    K.sum_duplicates()
    return K


def mass_fd(ns) -> sp.csr_matrix:
    return sp.identity(int(np.prod(ns)), format="csr")


def _q1_1d(n: int, h: float):
    M1 = _tridiag(n, h / 6.0, 4.0 * h / 6.0, h / 6.0)
    K1 = _tridiag(n, -1.0 / h, 2.0 / h, -1.0 / h)
    return M1, K1


def q1_matrices(ns, lens=None):
    """(M, K) for bilinear/trilinear elements on the tensor vertex mesh."""
    ns = tuple(int(n) for n in ns)
    hs = spacing(ns, lens)
    ones = [_q1_1d(n, h) for n, h in zip(ns, hs)]
    d = len(ns)
    # kron order: slowest axis first
    M = reduce(lambda X, Y: sp.kron(X, Y, format="csr"), [ones[a][0] for a in reversed(range(d))])
    K = None
    for a in range(d):
        facs = [ones[b][1] if b == a else ones[b][0] for b in reversed(range(d))]
        term = reduce(lambda X, Y: sp.kron(X, Y, format="csr"), facs)
        K = term if K is None else K + term
    return M.tocsr(), K.tocsr()


def _q2_1d(n: int, h: float):
    """1D quadratic Lagrange elements on n interior nodes of spacing h (n odd): (n + 1) / 2 elements
    of size H = 2h, nodes (left, midpoint, right).  Element matrices (exact integrals):
    mass H/30 [[4, 2, -1], [2, 16, 2], [-1, 2, 4]], stiffness 1/(3H) [[7, -8, 1], [-8, 16, -8],
    [1, -8, 7]]; assembled on all 2E + 1 nodes, then restricted to the interior ones."""
    if n % 2 != 1:
        raise ValueError("Q2 elements need an odd number of interior nodes per axis")
    E = (n + 1) // 2
    H = 2.0 * h
    Me = H / 30.0 * np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]])
    Ke = 1.0 / (3.0 * H) * np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]])
    N = 2 * E + 1
    M = np.zeros((N, N))
    K = np.zeros((N, N))
    for e in range(E):
        idx = [2 * e, 2 * e + 1, 2 * e + 2]
        M[np.ix_(idx, idx)] += Me
        K[np.ix_(idx, idx)] += Ke
    return sp.csr_matrix(M[1:-1, 1:-1]), sp.csr_matrix(K[1:-1, 1:-1])


def q2_matrices(ns, lens=None):
    """(M, K) for biquadratic/triquadratic elements on the tensor mesh whose interior nodes (element
    vertices and midpoints) are the vertex grid of `ns` (every n odd)."""
    ns = tuple(int(n) for n in ns)
    hs = spacing(ns, lens)
    ones = [_q2_1d(n, h) for n, h in zip(ns, hs)]
    d = len(ns)
    M = reduce(lambda X, Y: sp.kron(X, Y, format="csr"), [ones[a][0] for a in reversed(range(d))])
    K = None
    for a in range(d):
        facs = [ones[b][1] if b == a else ones[b][0] for b in reversed(range(d))]
        term = reduce(lambda X, Y: sp.kron(X, Y, format="csr"), facs)
        K = term if K is None else K + term
    return M.tocsr(), K.tocsr()


def q1_jacobi_interval(d: int):
    """Spectrum bounds of D^{-1} M for the Q1 mass matrix: [2^-d, (3/2)^d]."""
    return 0.5 ** d, 1.5 ** d


def q2_jacobi_interval(d: int):
    """Spectrum bounds of D^{-1} M for the Q2 mass matrix: [2^-d, (5/4)^d].  Element by element
    (D = sum of the element diagonals), the 1D element pencil diag(M_e)^{-1} M_e has eigenvalues
    1/2, 5/4, 5/4; the tensor product multiplies the 1D bounds."""
    return 0.5 ** d, 1.25 ** d


def operators(ns, lens=None, disc: str = "fd", kappa=None):
    """Return (M, K) as CSR; M is None to mean the identity (FD)."""
    if disc == "fd":
        return None, stiffness_fd(ns, lens, kappa)
    if disc in ("q1", "q2"):
        if kappa is not None:
            raise ValueError("variable kappa is only defined for the FD discretisation")
        return q1_matrices(ns, lens) if disc == "q1" else q2_matrices(ns, lens)
    raise ValueError(disc)
