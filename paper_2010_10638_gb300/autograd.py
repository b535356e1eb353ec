"""torch.autograd.Function over libtucker's adjoint (tucker_loss_grad).

    loss = TuckerLoss.apply(ctx, G, U_1, ..., U_N)

is the observed-entry loss 1/2 sum_z (x_z - [[G; U_1..U_N]]_z)^2 over the nonzeros
held by the tucker context `ctx`, in FP32 (loss accumulated in FP64).  The forward
call already runs the adjoint kernels (the gradients come from the same residuals),
so backward only scales the saved gradients by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import tucker as T


class TuckerLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, G, *U):
        loss, dU, dG = T.tucker_loss_grad(ctx, list(U), G)
        fctx.save_for_backward(dG, *dU)
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad):
        dG, *dU = fctx.saved_tensors
        g = grad.to(torch.float32)
        return (None, g * dG, *[g * d for d in dU])


def tucker_loss(ctx, G, U):
    return TuckerLoss.apply(ctx, G, *U)
