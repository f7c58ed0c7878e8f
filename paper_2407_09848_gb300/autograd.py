"""torch.autograd wrappers of the smoother and the V-cycle.

Forward and backward both run in libamgps kernels (amgps_smooth /
amgps_smooth_backward, amgps_vcycle / amgps_vcycle_backward); these classes
only connect them to torch's autograd.  Weights are CPU float64 tensors (they
are scalars per level, set on the library context before each call).
"""
from __future__ import annotations

import numpy as np
import torch


class SmootherFn(torch.autograd.Function):
    """x = S(b, x0; beta) on one level with the AMGPS_WEIGHTS recurrence
    (Eq. polsmootheropt with learned beta)."""

    @staticmethod
    def forward(ctx, b, x0, beta, solver, level):
        k = int(beta.numel())
        solver.set_smoother(level, "weights", k, weights=beta.detach().cpu().numpy())
        x = x0.detach().clone().contiguous()
        solver.smooth(level, "weights", k, b.detach().contiguous(), x, x_is_zero=False)
        ctx.save_for_backward(b.detach(), x0.detach(), beta.detach())
        ctx.solver, ctx.level = solver, level
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x0, beta = ctx.saved_tensors
        k = int(beta.numel())
        ctx.solver.set_smoother(ctx.level, "weights", k, weights=beta.cpu().numpy())
        gb, gx0, gw = ctx.solver.smooth_backward(ctx.level, "weights", k, b.contiguous(),
                                                 x0.contiguous(), gx.contiguous())
        return gb, gx0, torch.from_numpy(gw).to(beta.dtype), None, None


class VCycleFn(torch.autograd.Function):
    """z = B(beta_0, ..., beta_{L-2}) r, one V-cycle with per-level learned
    weights (a (levels-1, k) CPU tensor)."""

    @staticmethod
    def forward(ctx, r, betas, solver):
        for l in range(betas.shape[0]):
            solver.set_smoother(l, "weights", betas.shape[1], weights=betas[l].detach().cpu().numpy())
        z = torch.empty_like(r)
        solver.vcycle(r.detach().contiguous(), z)
        ctx.save_for_backward(r.detach(), betas.detach())
        ctx.solver = solver
        return z

    @staticmethod
    def backward(ctx, gz):
        r, betas = ctx.saved_tensors
        S = ctx.solver
        for l in range(betas.shape[0]):
            S.set_smoother(l, "weights", betas.shape[1], weights=betas[l].cpu().numpy())
        gr, gw = S.vcycle_backward(r.contiguous(), gz.contiguous())
        k = betas.shape[1]
        return gr, torch.from_numpy(np.ascontiguousarray(gw[:, :k])).to(betas.dtype), None
