"""H -> H' as a differentiable operation.

Forward runs ``lfbp_backproject_array``; backward runs ``lfbp_adjoint``, the
adjoint gather (for the full transpose the map is its own inverse, Sec. 4,
so the gradient is moved, never summed: no atomics).  This lets a loss on
backprojected volumes be differentiated with respect to the PSF array H,
as iterative PSF updates (Sec. 3.1) would need.
"""
from __future__ import annotations

import torch

from . import _lib


class LFBackproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H: torch.Tensor, plan: "_lib.Plan"):
        ctx.plan = plan
        return _lib.backproject_array(plan, H.contiguous())

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        return _lib.adjoint(ctx.plan, grad_out.contiguous()), None


def backprojection_array(H: torch.Tensor, plan: "_lib.Plan") -> torch.Tensor:
    """Differentiable H -> H' for a flat ragged array ``H`` described by ``plan``."""
    return LFBackproject.apply(H, plan)


class LFBackprojectVolume(torch.autograd.Function):
    """g = H' f with f fixed; differentiable with respect to H'."""

    @staticmethod
    def forward(ctx, Hp: torch.Tensor, f: torch.Tensor, plan: "_lib.Plan"):
        f = f.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(f)
        return _lib.backproject_volume(plan, Hp.contiguous(), f)

    @staticmethod
    def backward(ctx, grad_g: torch.Tensor):
        (f,) = ctx.saved_tensors
        return _lib.backproject_volume_grad(ctx.plan, f, grad_g.contiguous()), None, None


def backproject_volume(Hp: torch.Tensor, f: torch.Tensor, plan: "_lib.Plan") -> torch.Tensor:
    """Differentiable (in H') backprojection g = H' f of a sensor image f [Wx, Wy]."""
    return LFBackprojectVolume.apply(Hp, f, plan)
