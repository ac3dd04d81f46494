"""Two-level multigrid reduction in time (MGRIT) for the time recurrence of S_tilde.

Test infrastructure only (see the package header).

Sec. 5: in the paper's parallel implementation the block forward substitution inside the Schur
approximation S_tilde (Eq. AppSchur) is replaced by an MGRIT routine (the XBraid library).  The
paper gives no MGRIT parameters.  The algorithm restated here is the two-level method of
Falgout, Friedhoff, Kolev, MacLachlan and Schroder (SIAM J. Sci. Comput. 36(6), 2014), applied
to a recurrence

    u_0 = w_0,   u_{n+1} = Phi(u_n) + w_{n+1}   (n = 0 .. nt-1),

where Phi is one step of the substitution (for S_tilde: Phi(z) = z - tau (b^T (x) I)
Theta_tilde^{-1} (e (x) K z)).  Phi may be nonlinear (inner GMRES with a tolerance is); the
method is used in its residual-correction form all the same.

Reading (the paper is silent):
* two levels; coarsening factor m (2 <= m <= nt); C-points the multiples of m up to nt, F-points the
  rest; where m does not divide nt the steps after the last C-point form a shorter final interval,
  relaxed from that C-point, and the coarse recurrence has nt // m steps (the convention of MGRIT
  codes, XBraid's among them: the coarse grid is every m-th fine point);
* initial guess u_0 = w_0 (exact) and u_n = 0 for n > 0;
* one iteration = relaxation ("F": F-relaxation; "FCF": F-, C-, F-relaxation), then the C-point
  residuals r_j = w_{jm} + Phi(u_{jm-1}) - u_{jm}, then the coarse error recurrence
  e_0 = 0, e_j = Phi_c(e_{j-1}) + r_j solved by substitution, then u_{jm} += e_j;
* after the last iteration a final F-relaxation makes every F-point consistent with its C-point;
* Phi_c, the coarse propagator, is supplied by the caller (for S_tilde: the same step with step
  size m tau, i.e. Theta_tilde and its multigrid rebuilt for the shifts m tau d_i).

`vcycle` / `multilevel` are the multilevel form (XBraid's default): the coarse error equation is
itself solved by one V-cycle, down to a level solved by substitution.

Parity: pinned (tests) by the exactness property of MGRIT -- after k iterations the first
(2k+1)m points (FCF) or (k+1)m points (F) equal sequential substitution, for any Phi_c with
Phi_c(0) = 0, whether or not m divides nt -- by one-iteration convergence with the ideal coarse propagator Phi_c = Phi^m for a
linear Phi (two levels) and Phi^m, Phi^(m^2) (three levels), by the coarse S_tilde step on sine
eigenmodes against the RK stability function R(-m tau lambda), and by the multilevel cycle with
two levels being the two-level method bit for bit.
"""
from __future__ import annotations

import numpy as np


def f_relax(phi, u, w, m):
    """u_{n+1} = Phi(u_n) + w_{n+1} for every F-point, interval by interval from its C-point."""
    nt = u.shape[0] - 1
    for c0 in range(0, nt, m):
        for n in range(c0, min(c0 + m, nt + 1) - 1):
            u[n + 1] = phi(u[n]) + w[n + 1]


def c_relax(phi, u, w, m):
    """u_{jm} = Phi(u_{jm-1}) + w_{jm} for every C-point but the first."""
    nt = u.shape[0] - 1
    for c in range(m, nt + 1, m):
        u[c] = phi(u[c - 1]) + w[c]


def two_level(phi, phi_c, w, m: int, iters: int = 1, relax: str = "FCF", u=None):
    """Approximate the solution of u_0 = w_0, u_{n+1} = Phi(u_n) + w_{n+1} by `iters` two-level
    MGRIT iterations.  w has shape (nt + 1, n); returns u of the same shape."""
    w = np.asarray(w, dtype=np.float64)
    nt = w.shape[0] - 1
    if m < 1 or m > max(nt, 1):
        raise ValueError("the coarsening factor must lie in 1 .. nt")
    if relax not in ("F", "FCF"):
        raise ValueError("relaxation is 'F' or 'FCF'")
    if u is None:
        u = np.zeros_like(w)
        u[0] = w[0]
    else:
        u = np.array(u, dtype=np.float64)
    nc = nt // m               # C-points m, 2m, .., nc m; the steps after nc m are F-points
    for _ in range(iters):
        f_relax(phi, u, w, m)
        if relax == "FCF":
            c_relax(phi, u, w, m)
            f_relax(phi, u, w, m)
        r = [w[j * m] + phi(u[j * m - 1]) - u[j * m] for j in range(1, nc + 1)]
        e = np.zeros_like(w[0])
        for j in range(1, nc + 1):
            e = phi_c(e) + r[j - 1]
            u[j * m] = u[j * m] + e
    f_relax(phi, u, w, m)
    return u


def sequential(phi, w):
    """The substitution itself: u_0 = w_0, u_{n+1} = Phi(u_n) + w_{n+1}."""
    w = np.asarray(w, dtype=np.float64)
    u = np.empty_like(w)
    u[0] = w[0]
    for n in range(w.shape[0] - 1):
        u[n + 1] = phi(u[n]) + w[n + 1]
    return u


def vcycle(phis, w, m: int, relax: str = "FCF", u=None):
    """One multilevel MGRIT V-cycle (Falgout et al. 2014) for u_0 = w_0, u_{n+1} = phis[0](u_n) +
    w_{n+1}.  phis[k] is the propagator of level k (step size m^k tau); level k has nt / m^k steps
    and the last level is solved by substitution.  On every other level: relaxation, the C-point
    residuals, one V-cycle for the coarse error equation e_0 = 0, e_j = phis[k+1](e_{j-1}) + r_j from
    a zero guess, the C-point correction u_{jm} += e_j and an F-relaxation (ideal interpolation).
    With two levels this is one iteration of `two_level` followed by its final F-relaxation."""
    w = np.asarray(w, dtype=np.float64)
    nt = w.shape[0] - 1
    if u is None:
        u = np.zeros_like(w)
        u[0] = w[0]
    else:
        u = np.array(u, dtype=np.float64)
    if len(phis) == 1:
        return sequential(phis[0], w)
    if m < 1 or nt % m != 0:
        raise ValueError("the coarsening factor must divide the number of time steps on every level")
    if relax not in ("F", "FCF"):
        raise ValueError("relaxation is 'F' or 'FCF'")
    phi = phis[0]
    nc = nt // m
    f_relax(phi, u, w, m)
    if relax == "FCF":
        c_relax(phi, u, w, m)
        f_relax(phi, u, w, m)
    r = np.zeros((nc + 1,) + w.shape[1:])
    for j in range(1, nc + 1):
        r[j] = w[j * m] + phi(u[j * m - 1]) - u[j * m]
    e = vcycle(phis[1:], r, m, relax)
    for j in range(1, nc + 1):
        u[j * m] = u[j * m] + e[j]
    f_relax(phi, u, w, m)
    return u


def multilevel(phis, w, m: int, iters: int = 1, relax: str = "FCF"):
    """`iters` multilevel V-cycles from the zero guess (u_0 = w_0)."""
    u = None
    for _ in range(iters):
        u = vcycle(phis, w, m, relax, u)
    return u
