"""torch.autograd.Function over the all-at-once solve: forward = aao_rk_solve,
backward = aao_rk_adjoint_solve (the transposed all-at-once system solved with
the transposed preconditioner, backward in time).

x = HeatSolve.apply(f, u0, kappa, cfg) returns the space-time solution
[v_0..v_nt ; V] for the constant-in-time source f and initial data u0 on the
finite-difference grid of cfg; gradients flow to f, u0 and the nodal kappa.

Checkpointing (cfg["ckpt_every"] = k > 0): the forward pass keeps only the
states v_0, v_k, v_2k, ... instead of the whole space-time trajectory.  The
adjoint solve needs no forward state; the kappa gradient does (through
W_{n,i} = v_n + tau sum_j a_ij V_{n,j}), so backward recomputes each window
of k steps by an all-at-once solve started from its checkpoint and sums the
window contributions with aao_rk_grad_kappa(accumulate=1).
"""
from __future__ import annotations

import torch

from .api import Solver


def _window_solver(cache, cfg, kappa, nt_w):
    if nt_w not in cache:
        c = dict(cfg)
        c["nt"] = nt_w
        c["T"] = cfg["T"] * nt_w / cfg["nt"]          # same step tau
        # the recomputed window must reach the forward solve's tolerance (a window that stops short
        # raises), so it may take more outer iterations than the forward solve's cap
        c["maxit"] = max(cfg.get("maxit", 100), 200)
        m = int(c.get("mgrit_m", 0) or 0)
        c["mgrit_m"] = m if 1 < m < nt_w else 0    # MGRIT only where a window has two or more intervals
        cache[nt_w] = Solver(kappa=kappa, **c)
    return cache[nt_w]


class HeatSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, u0, kappa, cfg):
        cfg = dict(cfg)
        if cfg.get("disc", "fd") != "fd":
            raise NotImplementedError("the autograd wrapper covers the finite-difference grid (M = I)")
        k = int(cfg.pop("ckpt_every", 0) or 0)
        kap = None if kappa is None else kappa.detach().contiguous()
        S = Solver(kappa=kap, **cfg)
        x = torch.zeros(S.n_st, dtype=torch.float64, device=f.device)
        _, info = S.solve(f.detach().contiguous(), u0.detach().contiguous(), x)
        ctx.S, ctx.cfg, ctx.k, ctx.kap = S, cfg, k, kap
        ctx.has_kappa = kappa is not None
        ctx.info = info
        ctx.f = f.detach().contiguous()
        if k > 0 and k < S.nt:
            # keep v_0, v_k, v_2k, ... and v_nt (the tracked final state)
            idx = list(range(0, S.nt, k)) + [S.nt]
            ctx.ckpt_idx = idx
            ctx.save_for_backward(torch.stack([x[n * S.nx:(n + 1) * S.nx] for n in idx]).clone())
            ctx.full = False
        else:
            ctx.save_for_backward(x)
            ctx.full = True
        return x

    @staticmethod
    def backward(ctx, gx):
        (saved,) = ctx.saved_tensors
        S = ctx.S
        dev = gx.device
        lam = torch.zeros(S.n_st, dtype=torch.float64, device=dev)
        gf = torch.zeros(S.nx, dtype=torch.float64, device=dev)
        gk = None
        if ctx.has_kappa:
            nnode = 1
            for v in S.n:
                nnode *= v + 2
            gk = torch.zeros(nnode, dtype=torch.float64, device=dev)
        if ctx.full or not ctx.has_kappa:
            S.adjoint_solve(gx.contiguous(), lam, x_fwd=saved if ctx.has_kappa else None, grad_f=gf,
                            grad_kappa=gk)
        else:
            S.adjoint_solve(gx.contiguous(), lam, grad_f=gf)
            nx, nt, s, k = S.nx, S.nt, S.s, ctx.k
            cache = {}
            lv = lam[: (nt + 1) * nx]
            lV = lam[(nt + 1) * nx:]
            for w, n0 in enumerate(ctx.ckpt_idx[:-1]):
                nw = min(k, nt - n0)
                Sw = _window_solver(cache, ctx.cfg, ctx.kap, nw)
                xw = torch.zeros(Sw.n_st, dtype=torch.float64, device=dev)
                Sw.solve(ctx.f, saved[w].contiguous(), xw)
                lamw = torch.cat([lv[n0 * nx:(n0 + nw + 1) * nx], lV[n0 * s * nx:(n0 + nw) * s * nx]]).contiguous()
                Sw.grad_kappa(lamw, xw, gk, accumulate=True)
            for Sw in cache.values():
                Sw.close()
        gu0 = lam[: S.nx].clone()          # M^T lambda_{v,0}, M = I (FD)
        return gf, gu0, gk, None


def heat_solve(f, u0, kappa=None, **cfg):
    return HeatSolve.apply(f, u0, kappa, cfg)
