"""torch.autograd wrapper of the forward map.

``fwd_model(problem, m)`` returns the receiver data f(m) (paper eq. (data));
its backward applies the migration operator F* (eq. (grad)) to the incoming
data gradient and its forward-mode derivative applies the Born operator F.
Any torch loss on the data then gets the adjoint-state gradient, e.g. the
misfit of section 2.1, Phi = 1/(2 sigma^2) |f(m) - d_obs|^2, whose gradient is
F* (f(m) - d_obs) / sigma^2.  The Gauss-Newton Hessian action is its own op
(``Problem.hessian_apply``); it is not obtained by double differentiation.
"""
from __future__ import annotations

import torch

from .hv import HV_CKPT_ALL

__all__ = ["FwdModel", "fwd_model", "misfit"]


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


def misfit(problem, m: torch.Tensor, d_obs: torch.Tensor, ckpt: int = HV_CKPT_ALL) -> torch.Tensor:
    """Phi(m) = 1/(2 sigma^2) sum (f(m) - d_obs)^2 as a differentiable FP64 scalar."""
    r = fwd_model(problem, m, ckpt).to(torch.float64) - d_obs.to(torch.float64)
    return 0.5 * (r * r).sum() / (problem.sigma ** 2)
