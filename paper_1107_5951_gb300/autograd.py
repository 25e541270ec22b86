"""PyTorch autograd wrapper of the forward model and its hand-written adjoint.

``gravity(rho, plan, component)`` returns g_z (``component="gz"``, shape
(B?, M)) or g (``"g"``, shape (B?, M, 3)) for densities rho on the plan's
grid; its backward calls ``gf_adjoint`` -- the transposed FMM (or the
transposed direct sum) -- so d(misfit)/d(rho) never differentiates through
the kernels.
"""
from __future__ import annotations

import torch


class GravityForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, plan, component="gz"):
        if component not in ("gz", "g"):
            raise ValueError("component must be 'gz' or 'g'")
        g, gz = plan.forward(rho, want_g=component == "g", want_gz=component == "gz")
        ctx.plan = plan
        ctx.component = component
        ctx.rho_dtype = rho.dtype
        return gz if component == "gz" else g

    @staticmethod
    def backward(ctx, grad_out):
        ncomp = 1 if ctx.component == "gz" else 3
        grad = ctx.plan.adjoint(grad_out.to(torch.float64).contiguous(), ncomp=ncomp)
        return grad.to(ctx.rho_dtype), None, None


def gravity(rho, plan, component="gz"):
    """g_z or g of the densities `rho` (CUDA tensor, (nz,ny,nx) or
    (B,nz,ny,nx)), differentiable with respect to `rho`."""
    return GravityForward.apply(rho, plan, component)
