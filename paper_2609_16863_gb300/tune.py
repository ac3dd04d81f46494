"""Schedule autotuner: choose how S_tilde's time recurrence runs for one problem.

The recurrence runs as the forward substitution of Eq. (AppSchur) (mgrit_m = 0) or as one
two-level MGRIT iteration with coarsening factor m (the parallel implementation of Sec. 5).
Which is faster depends on the problem: MGRIT does about twice the work of the substitution but
cuts its dependency chain from nt steps to about 2m + nt/m, which pays where a single step is
latency-bound (2D grids, whose shifted solves run on one thread-block cluster) and not where one
step already fills the GPU (large 3D grids).  `tune_mgrit` times one application of P_tilde per
candidate through the C ABI (after one untimed application that captures the step graphs) and
returns the fastest candidate with every timing.  One MGRIT iteration only approximates S_tilde's
recurrence, which can cost outer iterations (measured on 96^3 Gauss s = 2: 13 outer iterations with the
substitution, 18 with MGRIT m = 4), so MGRIT is taken only when it is at least `margin` (default 10%)
faster per application than the substitution.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional, Sequence, Tuple

from .api import Solver


def mgrit_candidates(nt: int, factors: Iterable[int] = (4, 6, 8, 9, 10, 11, 12, 16, 32)) -> list:
    """0 (substitution) and every factor m with at least two C-point intervals (m need not divide
    nt: the steps after the last C-point form a shorter final interval)."""
    return [0] + [m for m in factors if nt // m >= 2]


def tune_mgrit(n: Sequence[int], T: float, nt: int, candidates: Optional[Iterable[int]] = None,
               device: str = "cuda:0", margin: float = 0.1, **solver_kw) -> Tuple[int, Dict[int, float]]:
    """Return (chosen mgrit_m, {mgrit_m: ms per P_tilde application}) for the problem (n, T, nt) with
    the solver options solver_kw (precision, tableau, inner settings...): the fastest candidate, but
    the substitution (0) unless an MGRIT candidate is faster than it by more than `margin`."""
    import torch
    cands = list(candidates) if candidates is not None else mgrit_candidates(nt)
    times: Dict[int, float] = {}
    for m in cands:
        S = Solver(n, T, nt, mgrit_m=m, **solver_kw)
        g = torch.Generator(device=device).manual_seed(11)
        r = torch.randn(S.n_st, dtype=torch.float64, device=device, generator=g)
        z = torch.zeros_like(r)
        S.precond_apply(r, z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        S.precond_apply(r, z)
        e1.record()
        torch.cuda.synchronize()
        times[m] = e0.elapsed_time(e1)
        S.close()
        del r, z
    best = min(times, key=times.get)
    if best != 0 and 0 in times and times[best] > (1.0 - margin) * times[0]:
        best = 0
    return best, times
