"""torch.autograd.Function wrappers of the targets' CUDA forward/backward.

The forward launches the library's log-density kernel, which also produces
the hand-written gradient; the backward scales that gradient by the incoming
grad_output.  No torch arithmetic computes log p or its gradient.
"""
from __future__ import annotations

import torch

from .laps import Target


class TargetLogp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, target: Target) -> torch.Tensor:
        logp, grad = target.logp_grad(x.detach().contiguous())
        ctx.save_for_backward(grad)
        return logp

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad_out.unsqueeze(1) * grad, None


def target_logp(x: torch.Tensor, target: Target) -> torch.Tensor:
    """log p of each row of x (FP32, CUDA), differentiable in x."""
    return TargetLogp.apply(x, target)
