"""torch.autograd wrappers of the forward map and of the misfit.

``fwd_model(problem, m)`` returns the receiver data f(m) (paper eq. (data));
its backward applies the migration operator F* (eq. (grad)) to the incoming
data gradient and its forward-mode derivative applies the Born operator F.

``misfit(problem, m, d_obs)`` returns the misfit of section 2.1,
Phi = 1/(2 sigma^2) |f(m) - d_obs|^2, as an FP64 scalar.  The library forms
the residual, the FP64 sum and the gradient F* (f(m) - d_obs) / sigma^2 in one
call (hv_misfit_grad: one forward sweep, one adjoint sweep); the backward hands
that gradient on, scaled by the incoming gradient of Phi.  When m does not
require a gradient, the forward calls hv_misfit (forward sweep only).  d_obs is
treated as a constant.  The Gauss-Newton Hessian action is its own op
(``Problem.hessian_apply``); it is not obtained by double differentiation.
"""
from __future__ import annotations

import torch

from .hv import HV_CKPT_ALL

__all__ = ["FwdModel", "Misfit", "fwd_model", "misfit"]


class FwdModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, problem, ckpt: int):
        ctx.problem = problem
        ctx.ckpt = ckpt
        ctx.save_for_backward(m)
        ctx.m_point = m.detach()        # the linearisation point for forward mode
        return problem.fwd_model(m.detach().contiguous())

    @staticmethod
    def backward(ctx, grad_d: torch.Tensor):
        (m,) = ctx.saved_tensors
        g = ctx.problem.migrate(m.detach().contiguous(), grad_d.detach().to(torch.float32).contiguous(),
                                ckpt=ctx.ckpt)
        return g, None, None

    @staticmethod
    def jvp(ctx, dm: torch.Tensor, _p, _c):
        return ctx.problem.born(ctx.m_point.contiguous(), dm.detach().contiguous().unsqueeze(0))[0]


def fwd_model(problem, m: torch.Tensor, ckpt: int = HV_CKPT_ALL) -> torch.Tensor:
    """Differentiable f(m): data [ns, nt, nr] of the problem for velocity m [nz, nx]."""
    return FwdModel.apply(m, problem, ckpt)


class Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, problem, d_obs: torch.Tensor, ckpt: int):
        m32 = m.detach().contiguous()
        d32 = d_obs.detach().to(torch.float32).contiguous()
        if ctx.needs_input_grad[0]:
            phi, g = problem.misfit_grad(m32, d32, ckpt=ckpt)
            ctx.save_for_backward(g)
        else:
            phi = problem.misfit(m32, d32)
        return phi

    @staticmethod
    def backward(ctx, grad_phi: torch.Tensor):
        (g,) = ctx.saved_tensors
        return (g * grad_phi).to(g.dtype), None, None, None


def misfit(problem, m: torch.Tensor, d_obs: torch.Tensor, ckpt: int = HV_CKPT_ALL) -> torch.Tensor:
    """Phi(m) = 1/(2 sigma^2) sum (f(m) - d_obs)^2 as a differentiable FP64 scalar (hv_misfit_grad)."""
    return Misfit.apply(m, problem, d_obs, ckpt)
