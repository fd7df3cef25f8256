"""torch.autograd.Function around the hand-written hex8 internal force and its VJP kernel.

Forward: f = f_int(u; lambda_e, mu_e) (osam_hex8_force).  Backward: the library's VJP kernel gives
(df/du)^T g and the per-element cotangents of lambda_e and mu_e (osam_hex8_force_vjp).  Tensors are
CUDA float64, u and f of shape [nodes, 3], lambda_e and mu_e of shape [elements].
"""
from __future__ import annotations

import torch

from . import osam


class Hex8Force(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, lam_e, mu_e, dims, h, material):
        u = u.contiguous()
        lam_e = lam_e.contiguous()
        mu_e = mu_e.contiguous()
        f = torch.empty_like(u)
        osam.hex8_force(dims, h, material, 0.0, 0.0, u, f, lam_e=lam_e, mu_e=mu_e,
                        stream=torch.cuda.current_stream(u.device))
        ctx.save_for_backward(u, lam_e, mu_e)
        ctx.dims, ctx.h, ctx.material = dims, h, material
        return f

    @staticmethod
    def backward(ctx, g):
        u, lam_e, mu_e = ctx.saved_tensors
        g = g.contiguous()
        ub = torch.empty_like(u)
        lb = torch.empty_like(lam_e)
        mb = torch.empty_like(mu_e)
        osam.hex8_force_vjp(ctx.dims, ctx.h, ctx.material, 0.0, 0.0, u, g, ub, lb, mb, lam_e=lam_e, mu_e=mu_e,
                            stream=torch.cuda.current_stream(u.device))
        return ub, lb, mb, None, None, None


def hex8_force(u, lam_e, mu_e, dims, h, material="nh"):
    return Hex8Force.apply(u, lam_e, mu_e, tuple(dims), float(h), material)
