"""The ST-AGM data-fidelity loss as a differentiable PyTorch function.

loss(u, w) = sum_j sum_k g_eps((F(w o S_j u))_k; f_jk)      (sections 2.2, 2.4)

Forward and backward both run in libod2p.so: the forward computes the loss
only; the backward recomputes the exit waves F(w o S_j u) from u and w and
applies the hand-written adjoint (gradient of eq. objgrad pulled back through
F^* and S_j^T), so no J x m x m tensor of exit waves is kept between the two
passes.  Gradients follow PyTorch's convention for real losses of complex
tensors, d/dRe + i d/dIm, so torch.optim steps on u and w directly.
"""
from __future__ import annotations

import torch

from .api import Plan, stagm_loss_grad


class STAGMLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, w: torch.Tensor, plan: Plan) -> torch.Tensor:
        loss, _, _ = stagm_loss_grad(plan, u.detach().contiguous(), w.detach().contiguous(),
                                     grad_u=False, grad_w=False)
        ctx.plan = plan
        ctx.save_for_backward(u, w)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        u, w = ctx.saved_tensors
        need_u, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        _, gu, gw = stagm_loss_grad(ctx.plan, u.detach().contiguous(), w.detach().contiguous(),
                                    grad_u=need_u, grad_w=need_w)
        g = grad_out.to(torch.float32)
        return (gu * g if need_u else None), (gw * g if need_w else None), None


def stagm_loss(u: torch.Tensor, w: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable ST-AGM loss of image u (img_h x img_w) and probe w (m x m)."""
    return STAGMLoss.apply(u, w, plan)
