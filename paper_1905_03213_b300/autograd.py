"""Differentiable W-projection forward model: image -> grid -> visibilities.

The model visibilities of a real sky image X (N x N float32) are

    V = degrid(image_to_grid(X)),

image_to_grid being the adjoint of the imaging transform (taper division, then the centred
forward 2D DFT; sum of weights 1) and degrid the adjoint of gridding (Sec. 2 of Lao et al.
2019 names the two as the pair being accelerated). The map is linear, so its vector-Jacobian
product is its adjoint applied to the incoming gradient:

    dL/dX = Re(A^H g) = fft_to_image(grid(g, unit weights), sum_w = 1, taper-corrected),

with g the gradient with respect to V (torch's convention for complex outputs). The backward
pass therefore re-grids the incoming visibility gradient into a fresh grid: nothing of the
forward pass is kept but the coordinates' inputs (uvw, freq). Every step runs in libwproj's
kernels; this module only wires the calls into torch.autograd.
"""
from __future__ import annotations

import torch

from ._abi import WProj


class DegridImage(torch.autograd.Function):
    """V = degrid(image_to_grid(X)) for a real image X; backward = grid + image transform."""

    @staticmethod
    def forward(ctx, image: torch.Tensor, wp: WProj, uvw: torch.Tensor, freq: torch.Tensor) -> torch.Tensor:
        x = image.detach().to(torch.float32).contiguous()
        grid = wp.image_to_grid(x, sum_w=None, taper_correct=True)
        vis = wp.degrid(uvw, freq, grid)
        ctx.wp = wp
        ctx.save_for_backward(uvw, freq)
        return vis

    @staticmethod
    def backward(ctx, grad_vis: torch.Tensor):
        uvw, freq = ctx.saved_tensors
        wp: WProj = ctx.wp
        g = grad_vis.to(torch.complex64).contiguous()
        grid, _, _ = wp.grid(uvw, freq, g, None)
        one = torch.ones(1, dtype=torch.float64, device=g.device)
        grad_image = wp.fft_to_image(grid, one, taper_correct=True)
        return grad_image, None, None, None


def predict(wp: WProj, image: torch.Tensor, uvw: torch.Tensor, freq: torch.Tensor) -> torch.Tensor:
    """Model visibilities [nrow, nchan] complex64 of `image` [N, N]; differentiable in `image`."""
    return DegridImage.apply(image, wp, uvw, freq)
