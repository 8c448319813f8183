"""CP decomposition entry points on top of the engine (argument marshalling only).

``CPLoss`` is a ``torch.autograd.Function`` for the CP least-squares loss on the
observed entries, L = 1/2 sum_e (m_e - x_e)^2 with m_e = sum_r prod_k
A_k[i_k(e), r]: its forward is the engine's sampled CP reconstruction
(``cp_loss_fwd``) and its backward the engine's all-mode spMTTKRP of the
residuals (``cp_loss_bwd``).  ``cp_als`` runs CP-ALS iterations
(``cp_als_iter``, replayed as a CUDA graph).
"""
from __future__ import annotations

from typing import List, Sequence

import torch

from .binding import Plan


class CPLoss(torch.autograd.Function):
    """The plan holds the residuals of its latest forward only.  Each forward
    records the plan's loss generation; a backward whose forward is no longer
    the latest (another forward ran since, or an earlier backward consumed the
    residuals) first recomputes its residuals from its saved factors."""

    @staticmethod
    def forward(ctx, plan: Plan, *factors):
        fs = [f.contiguous() for f in factors]
        loss = torch.empty((), device=fs[0].device, dtype=torch.float32)
        ctx.generation = plan.loss_fwd(fs, loss)
        ctx.plan = plan
        ctx.save_for_backward(*fs)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        fs = ctx.saved_tensors
        if ctx.plan.loss_generation != ctx.generation:
            scratch = torch.empty((), device=fs[0].device, dtype=torch.float32)
            ctx.plan.loss_fwd(fs, scratch)
        grads = [torch.empty(f.shape, device=f.device, dtype=torch.float32) for f in fs]
        g = grad_out.detach().to(torch.float32).contiguous().reshape(())
        ctx.plan.loss_bwd(fs, g, grads)
        return (None, *[gr if f.dtype == torch.float32 else gr.to(f.dtype)
                        for gr, f in zip(grads, fs)])


def cp_loss(plan: Plan, factors: Sequence[torch.Tensor]) -> torch.Tensor:
    return CPLoss.apply(plan, *factors)


def cp_als(plan: Plan, factors: List[torch.Tensor], iters: int, tol: float = 0.0):
    """Runs up to ``iters`` CP-ALS iterations in place; returns (lambda, fits)."""
    lam = torch.empty(plan.rank, device=factors[0].device, dtype=torch.float32)
    fits = []
    for _ in range(int(iters)):
        fits.append(plan.als_iter(factors, lam))
        if tol > 0 and len(fits) > 1 and abs(fits[-1] - fits[-2]) < tol:
            break
    return lam, fits
