"""Differentiable additive-kernel product for PyTorch: y = K(points, ell, sigma_f) v.

The forward pass is addker_matvec; the backward pass is addker_vjp, hand-written kernels that give
the gradient of w^T K v (w the incoming gradient) with respect to v, every ell_s, sigma_f and the
point coordinates, for the operator as the NFFT fast summation computes it (Sec. 3.1, 3.3). The
backward recomputes the grids of v instead of keeping them from the forward pass, so a product costs
no memory beyond its plan between forward and backward.
"""
from __future__ import annotations

import torch

from . import AddKer


class _AdditiveKernelMatvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, points, ell, sigma_f, windows, bandwidth, cutoff, plan_kwargs):
        ell_list = [float(e) for e in ell.detach().cpu().tolist()]
        op = AddKer(points.detach().contiguous(), windows, ell_list, float(sigma_f), bandwidth, cutoff, **plan_kwargs)
        y = op.matvec(v.detach().contiguous())
        ctx.op = op
        ctx.save_for_backward(v)
        ctx.d = points.shape[1]
        return y

    @staticmethod
    def backward(ctx, grad_y):
        (v,) = ctx.saved_tensors
        op = ctx.op
        gv, gt, gx = op.vjp(v.detach().contiguous(), grad_y.detach().contiguous().to(torch.float32))
        P = op.P
        g_ell = gt[:P].to(torch.float32) if ctx.needs_input_grad[2] else None
        g_sf = gt[P].to(torch.float32) if ctx.needs_input_grad[3] else None
        op.close()
        ctx.op = None
        return (gv if ctx.needs_input_grad[0] else None, gx if ctx.needs_input_grad[1] else None,
                g_ell, g_sf, None, None, None, None)


def additive_kernel_matvec(points, v, ell, sigma_f, windows, bandwidth=32, cutoff=4, **plan_kwargs):
    """K v for the additive Gaussian kernel over `windows`, differentiable in v, points (N x d float32
    CUDA tensor, scaled into the ball of radius 1/4 - eps_B/2), ell (P-vector tensor) and sigma_f
    (0-d tensor)."""
    if not torch.is_tensor(ell):
        ell = torch.tensor(ell, dtype=torch.float32, device=points.device)
    if not torch.is_tensor(sigma_f):
        sigma_f = torch.tensor(float(sigma_f), dtype=torch.float32, device=points.device)
    return _AdditiveKernelMatvec.apply(v, points, ell, sigma_f, [tuple(w) for w in windows], bandwidth, cutoff,
                                       plan_kwargs)
