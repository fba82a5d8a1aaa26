"""PyTorch autograd over the C-ABI rasteriser.

`render(params, step)` returns the rendered images V x 3 x H x W of the step's
views as a differentiable function of the parameter matrix (rows x n_pad):
the forward pass is projection, binning and alpha blending; the backward pass
hands the incoming image gradient to the reverse pass as its cotangent
(GS_LOSS_COTANGENT) and returns J^T grad_image.  The reverse pass recovers each
T_i from the pixel's final transmittance (nothing per pair is stored), so the
memory of a render is its records, pairs and images at any scene size.

`gn_diagonal(params, weights, step, t)` is the Hutchinson estimate of the
diagonal of the Gauss-Newton matrix J^T diag(weights) J at params (Sec. 4.1),
for a per-pixel weight image (for the L1 objective of Sec. 3.2,
weights = 1 / (4 max(|r|, delta)) / m), as a torch.autograd.Function: the
library renders with the probe tangents J z_k and its reverse pass forms
weights * J z_k and J^T of it itself (GS_LOSS_WEIGHTED).  The estimate enters
the optimiser's update as a constant (Algorithm 1 does not differentiate D_t),
so the Function's output carries no gradient.
"""
from __future__ import annotations

import torch

from .engine import TRStep


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, step: TRStep) -> torch.Tensor:
        if params.data_ptr() != step.x.data_ptr():
            step.x.copy_(params.detach())
        step.project(None, probes=False)
        step.bin_sort()
        step.raster_fwd(None, probes=False)
        ctx.step = step
        return step.image.view(step.V, 3, step.H, step.W).clone()

    @staticmethod
    def backward(ctx, grad_image: torch.Tensor):
        step = ctx.step
        cot = grad_image.detach().to(torch.float32).contiguous().view(-1)
        step.raster_bwd_cotangent(cot, None, True)
        return step.grad.clone(), None


def render(params: torch.Tensor, step: TRStep) -> torch.Tensor:
    """Differentiable render of `step`'s views (see the module text).  The step's
    cameras select the views; its records, pairs and images are overwritten."""
    return _Render.apply(params, step)


class _GNDiagonal(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, weights: torch.Tensor, step: TRStep, t: int) -> torch.Tensor:
        if params.data_ptr() != step.x.data_ptr():
            step.x.copy_(params.detach())
        step.project(t, probes=True)
        step.bin_sort()
        step.raster_fwd(t, probes=True)
        w = weights.detach().to(torch.float32).contiguous().view(-1)
        step.hvp_weighted(t, w)
        out = step.hz.clone()
        ctx.mark_non_differentiable(out)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        return None, None, None, None


def gn_diagonal(params: torch.Tensor, weights: torch.Tensor, step: TRStep, t: int) -> torch.Tensor:
    """Hutchinson estimate (step.nu probes of step t) of diag(J^T diag(w) J) at
    params for the weight image w (V x 3 x H x W): one render with the probe
    tangents and one reverse pass that weights and pulls back J z_k, both in the
    library.  step's records, pairs, images and hz are overwritten."""
    return _GNDiagonal.apply(params, weights, step, t)
