"""The time-reversal adjoint as a torch.autograd.Function.

`fwi_misfit(c, plan, weights, observed)` returns the misfit (mean over the K
encoded super-shots of D_k = 0.5 ||f_k - f_obs_k||^2, Eq. 8 with the encoded
estimator of Sec. 3.2) as a differentiable FP64 scalar of the sound speed c.
Its forward pass runs fwi_gradient, which computes the misfit and, by the
adjoint-state method with the time-reversed re-simulation (Alg. 1), the
gradient in the same call; backward returns grad_output times that gradient.

With a plan created with pairing="exact" and c_rec set to the receivers' sound
speed, the gradient is the derivative of the discrete misfit (up to the PML,
whose multipliers are not transposed by the scheme used for the adjoint).
"""
from __future__ import annotations

import torch

from . import fwi


class FwiMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, plan, weights, observed, encoded=True):
        if not c.is_cuda:
            raise ValueError("c must be a CUDA tensor")
        c32 = c.detach().to(torch.float32).contiguous().reshape(-1)
        misfit, grad = plan.gradient(c32, weights.contiguous(), observed.contiguous(), encoded=encoded)
        st = plan.status()
        if st != fwi.FWI_OK:
            raise fwi.FwiError(st, "fwi_gradient")
        ctx.save_for_backward(grad)
        ctx.c_shape, ctx.c_dtype = c.shape, c.dtype
        return misfit.mean()

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        g = (grad_output.to(torch.float64) * grad).reshape(ctx.c_shape).to(ctx.c_dtype)
        return g, None, None, None, None


def fwi_misfit(c, plan, weights, observed, encoded=True):
    """Differentiable misfit of sound speed c (see module docstring)."""
    return FwiMisfit.apply(c, plan, weights, observed, encoded)


class FwiLoss(torch.nn.Module):
    """Module form: holds a plan, the encoding weights and the observed data."""

    def __init__(self, plan, weights, observed, encoded=True):
        super().__init__()
        self.plan = plan
        self.register_buffer("weights", weights)
        self.register_buffer("observed", observed)
        self.encoded = encoded

    def forward(self, c):
        return fwi_misfit(c, self.plan, self.weights, self.observed, self.encoded)
