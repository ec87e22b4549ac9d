"""Degridding as a differentiable PyTorch operation.

``degrid(plan, image, uvw)`` returns the model visibilities of Algorithm 6
and back-propagates through the exact adjoint, the gridding of Algorithm 5
(Section 3.2: the degridding and gridding operators are adjoints of each
other, so the vector-Jacobian product of V = A f is A^H applied to the
incoming gradient).  Both directions run in the CUDA library; this module
only wires them into autograd.

A complex image gets the complex gradient A^H g (PyTorch's convention for
complex inputs); a real image gets its real part, which is the gradient of a
real loss with respect to a real sky.
"""
from __future__ import annotations

import torch

from .wstack import Plan


class DegridFunction(torch.autograd.Function):
    """V = A f with A the improved W-stacking degridder of ``plan``."""

    @staticmethod
    def forward(ctx, image: torch.Tensor, uvw: torch.Tensor, plan: Plan):
        ctx.plan = plan
        ctx.real_input = not image.is_complex()
        ctx.save_for_backward(uvw)
        img = torch.complex(image, torch.zeros_like(image)) if ctx.real_input else image
        vis = plan.degrid(img.contiguous(), uvw)
        ctx.vis_dtype = vis.dtype
        return vis

    @staticmethod
    def backward(ctx, grad_vis: torch.Tensor):
        (uvw,) = ctx.saved_tensors
        g = ctx.plan.grid(uvw, grad_vis.to(ctx.vis_dtype).contiguous())
        if ctx.real_input:
            g = g.real
        return g, None, None


def degrid(plan: Plan, image: torch.Tensor, uvw: torch.Tensor) -> torch.Tensor:
    """Differentiable degridding: visibilities of ``image`` at ``uvw`` (see DegridFunction).

    An optimisation loop calls this with the same uvw every step; binding it to
    the plan once (``plan.bind(uvw)``) lets the forward and backward calls skip
    the tap rule and the tile sort."""
    return DegridFunction.apply(image, uvw, plan)


def chi2(plan: Plan, image: torch.Tensor, uvw: torch.Tensor, target: torch.Tensor, sigma: float) -> torch.Tensor:
    """chi^2 = sum_k |V_k(image) - target_k|^2 / sigma^2, accumulated in float64."""
    r = degrid(plan, image, uvw) - target
    return (r.real.double() ** 2 + r.imag.double() ** 2).sum() / (sigma * sigma)
