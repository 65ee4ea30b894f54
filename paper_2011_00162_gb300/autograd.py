"""The ST-AGM data-fidelity loss as a differentiable PyTorch function.

loss(u, w) = sum_j sum_k g_eps((F(w o S_j u))_k; f_jk)      (sections 2.2, 2.4)

Forward and backward both run in libod2p.so.  The forward makes one pass over
the frames: exit wave, transform, loss and gradient frame h_j = F^* grad g_j
(the hand-written adjoint of eq. objgrad pulled back through F^*).  While the
J x m x m gradient frames fit in STORE_BUDGET_BYTES (8 GiB) the forward keeps them in
the plan (stagm_loss_grad with STORE) and the backward only gathers them into
the gradients (FROM_STORE); above the budget nothing is kept and the backward
recomputes the exit waves from u and w (RECOMPUTE).  Gradients follow
PyTorch's convention for real losses of complex tensors, d/dRe + i d/dIm, so
torch.optim steps on u and w directly.
"""
from __future__ import annotations

import torch

from ._lib import ERR_STATE
from .api import FROM_STORE, RECOMPUTE, STORE, Plan, PtychoError, stagm_loss_grad

# storing always took less time than recomputing (4096^2 / 6561 frames of 256^2: loss then
# gradient 6.9 ms stored against 12.3 ms recomputed, for 3.4 GB of frames), so the budget
# only bounds memory
STORE_BUDGET_BYTES = 8 << 30


def stores_frames(plan: Plan) -> bool:
    """Whether the forward keeps the gradient frames for the backward."""
    return plan.n_frames * plan.geom.m * plan.geom.m * 8 <= STORE_BUDGET_BYTES


class STAGMLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, w: torch.Tensor, plan: Plan) -> torch.Tensor:
        uc, wc = u.detach().contiguous(), w.detach().contiguous()
        ctx.stored = stores_frames(plan)
        loss, _, _ = stagm_loss_grad(plan, uc, wc, grad_u=False, grad_w=False,
                                     recompute=STORE if ctx.stored else RECOMPUTE)
        ctx.plan = plan
        ctx.ptrs = (uc.data_ptr(), wc.data_ptr())
        ctx.save_for_backward(uc, wc)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        u, w = ctx.saved_tensors
        need_u, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        done = False
        if ctx.stored and (u.data_ptr(), w.data_ptr()) == ctx.ptrs:
            try:  # the frames kept by this forward, unless a later forward replaced them
                _, gu, gw = stagm_loss_grad(ctx.plan, u, w, grad_u=need_u, grad_w=need_w, recompute=FROM_STORE)
                done = True
            except PtychoError as e:
                if e.code != ERR_STATE:
                    raise
        if not done:
            _, gu, gw = stagm_loss_grad(ctx.plan, u, w, grad_u=need_u, grad_w=need_w, recompute=RECOMPUTE)
        g = grad_out.to(torch.float32)
        return (gu * g if need_u else None), (gw * g if need_w else None), None


def stagm_loss(u: torch.Tensor, w: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable ST-AGM loss of image u (img_h x img_w) and probe w (m x m)."""
    return STAGMLoss.apply(u, w, plan)
