"""The FWIME objective as a torch.autograd.Function (Barnier et al., Eq. 1 at a
fixed extended perturbation p~, gradient Eqs. 7-9 with S = I).

forward(v) runs libfwime's gradient schedule -- the forward sweep (f + B~ p~,
residual, objective) followed by the hand-written adjoint kernels (Born adjoint
B* r and tomographic adjoint T* r, with checkpointed recomputation of the
source-side wavefields) -- in one call, because the adjoint sweep consumes the
forward sweep's checkpoints; backward() returns grad_output * (B* r + T* r).
When v does not require a gradient only the forward sweep runs.
"""
from __future__ import annotations

import torch


class FwimeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, context, w, pt, dobs, eps):
        if ctx.needs_input_grad[0]:
            grad = torch.empty_like(v)
            J = context.gradient(v.detach().contiguous(), w, pt, dobs, grad, eps=eps)
            ctx.save_for_backward(grad)
        else:
            J = context.objective(v.detach().contiguous(), w, pt, dobs, eps=eps)
        return torch.tensor(J, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ.to(grad.dtype) * grad, None, None, None, None, None)


def fwime_objective(context, v, w, pt, dobs, eps: float = 0.0):
    """Phi_eps(v) at fixed p~ as a differentiable scalar (float64)."""
    return FwimeObjective.apply(v, context, w, pt, dobs, float(eps))


class SplineParam(torch.autograd.Function):
    """v = S m: the model on a coarse spline grid interpolated onto the finite-difference grid (Eq. 1);
    backward applies S*, so a gradient on the FD grid becomes a gradient on the spline nodes."""

    @staticmethod
    def forward(ctx, m, context, zs, xs):
        g = context.grid
        v = torch.empty((g.nz, g.nx), dtype=torch.float32, device=m.device)
        context.spline(zs, xs, m.detach().contiguous(), v)
        ctx.context, ctx.zs, ctx.xs, ctx.shape = context, zs, xs, m.shape
        return v

    @staticmethod
    def backward(ctx, gv):
        gm = torch.empty(ctx.shape, dtype=torch.float32, device=gv.device)
        ctx.context.spline(ctx.zs, ctx.xs, gv.contiguous().to(torch.float32), gm, adjoint=True)
        return gm, None, None, None


def spline_param(context, zs, xs, m):
    """S m as a differentiable map from the spline nodes zs x xs (metres) to the context's grid."""
    return SplineParam.apply(m, context, zs, xs)
