"""Differentiable forms of the dose model and objective, on libvmat kernels.

``ApertureDose(ddc, mlc, cps, leaves)(y)`` is d(y) = D (A y): the dose of the
apertures ``cps``/``leaves`` at intensities y (Section 2.1, z = sum_k DA(A_k) y_k).
Its backward is the hand-written adjoint A^T D^T g_d: ``beamlet_price`` (Eq. 3's
D^T product) followed by ``aperture_grad`` (sum over each aperture's beamlets).

``objective(z, vox)`` is F(z) of Eq. 1 (float64 scalar); its backward is
-g(z) from Eq. 4, computed by ``objective_grad`` in the forward pass.

Composed, ``objective(ApertureDose(...)(y), vox)`` differentiates to
grad_y F = -A^T D^T g, the master problem's gradient (Eq. 6-8).
"""
from __future__ import annotations

import torch

from . import api


class _Dose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, h, mlc, cps, leaves, V, J):
        y = y.detach().contiguous()
        x = torch.empty(J, dtype=torch.float32, device=y.device)
        api.aperture_fluence(mlc, cps, leaves, y, x)
        d = torch.empty(V, dtype=torch.float32, device=y.device)
        api.dose_forward(h, x, d)
        ctx.h, ctx.mlc, ctx.J = h, mlc, J
        ctx.save_for_backward(cps, leaves)
        return d

    @staticmethod
    def backward(ctx, gd):
        cps, leaves = ctx.saved_tensors
        pi = torch.empty(ctx.J, dtype=torch.float32, device=gd.device)
        api.beamlet_price(ctx.h, gd.detach().to(torch.float32).contiguous(), pi)
        gy = torch.empty(cps.numel(), dtype=torch.float32, device=gd.device)
        api.aperture_grad(ctx.mlc, cps, leaves, pi, gy)
        return gy, None, None, None, None, None, None


class ApertureDose:
    """d(y) = D (A y) for a fixed set of apertures (CP indices and leaf pairs)."""

    def __init__(self, ddc: "api.Ddc", mlc, cps: torch.Tensor, leaves: torch.Tensor):
        self.ddc, self.mlc = ddc, mlc
        self.cps = cps.to(torch.int32).contiguous()
        self.leaves = leaves.to(torch.int16).contiguous().view(-1)

    def __call__(self, y: torch.Tensor) -> torch.Tensor:
        return _Dose.apply(y, self.ddc.h, self.mlc, self.cps, self.leaves, self.ddc.V, self.ddc.J)


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, vox):
        z = z.detach().contiguous()
        g = torch.empty_like(z)
        F = torch.empty(1, dtype=torch.float64, device=z.device)
        api.objective_grad(z, vox, g, F)
        ctx.save_for_backward(g)
        return F[0]

    @staticmethod
    def backward(ctx, gF):
        (g,) = ctx.saved_tensors
        return -g * gF.to(g.dtype), None


def objective(z: torch.Tensor, vox: "api.VoxelParams") -> torch.Tensor:
    """F(z) (Eq. 1) as a differentiable float64 scalar; dF/dz = -g (Eq. 4)."""
    return _Objective.apply(z, vox)
