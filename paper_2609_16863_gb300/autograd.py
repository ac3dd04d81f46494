"""torch.autograd.Function over the all-at-once solve: forward = aao_rk_solve,
backward = aao_rk_adjoint_solve (the transposed all-at-once system solved with
the transposed preconditioner, backward in time).

x = HeatSolve.apply(f, u0, kappa, cfg) returns the space-time solution
[v_0..v_nt ; V] for the constant-in-time source f and initial data u0 on the
FD grid of cfg; gradients flow to f, u0 and (when given) the nodal kappa.
"""
from __future__ import annotations

import torch

from .api import Solver


class HeatSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, u0, kappa, cfg):
        cfg = dict(cfg)
        S = Solver(kappa=None if kappa is None else kappa.detach().contiguous(), **cfg)
        x = torch.zeros(S.n_st, dtype=torch.float64, device=f.device)
        _, info = S.solve(f.detach().contiguous(), u0.detach().contiguous(), x)
        ctx.S = S
        ctx.has_kappa = kappa is not None
        ctx.kappa_numel = None if kappa is None else kappa.numel()
        ctx.info = info
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        S = ctx.S
        lam = torch.zeros_like(x)
        gf = torch.zeros(S.nx, dtype=torch.float64, device=x.device)
        gk = torch.zeros(ctx.kappa_numel, dtype=torch.float64, device=x.device) if ctx.has_kappa else None
        S.adjoint_solve(gx.contiguous(), lam, x_fwd=x, grad_f=gf, grad_kappa=gk)
        gu0 = lam[: S.nx].clone()          # M^T lambda_{v,0}, M = I
        return gf, gu0, gk, None


def heat_solve(f, u0, kappa=None, **cfg):
    return HeatSolve.apply(f, u0, kappa, cfg)
