"""torch.autograd bridge of the internal force: f(u) as a differentiable
function of the displacement, with the adjoint (vector-Jacobian) product of the
tangent kernel as its backward pass.

Forward is pd_force at u (no bond breaking), backward is pd_vjp linearised at
the same u: for a loss L, dL/du = K^T dL/df with K = df/du the matrix-free
tangent that replaces the assembled stiffness of Eq. (6). Both run in libpd;
this module only passes torch tensors (FP64, CUDA, shape (npoints, dim), user
order) to it on torch's current stream. PMB simulations only (the tangent
kernel's model).
"""
from __future__ import annotations

import torch

from . import pd


class InternalForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, sim: pd.Sim) -> torch.Tensor:
        u = u.contiguous()
        f = torch.empty_like(u)
        pd.pd_force(sim, u=u, f_out=f, stream=torch.cuda.current_stream())
        ctx.save_for_backward(u)
        ctx.sim = sim
        return f

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        (u,) = ctx.saved_tensors
        grad_u = torch.empty_like(u)
        pd.pd_vjp(ctx.sim, grad_f.contiguous(), u_lin=u, out=grad_u, stream=torch.cuda.current_stream())
        return grad_u, None


def internal_force(sim: pd.Sim, u: torch.Tensor) -> torch.Tensor:
    """f(u) with autograd support (FP64 CUDA tensor of shape (npoints, dim))."""
    if u.dtype != torch.float64 or not u.is_cuda:
        raise ValueError("u must be a float64 CUDA tensor")
    return InternalForce.apply(u, sim)
