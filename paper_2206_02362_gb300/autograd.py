"""The FWIME objective as a torch.autograd.Function (Barnier et al., Eq. 1 at a
fixed extended perturbation p~, gradient Eqs. 7-9 with S = I).

forward(v) runs libfwime's forward sweep only (fwime_gradient_forward): f +
B~ p~, the residual and Phi, keeping the checkpoints of the source-side
wavefields and the residual in the context.  backward() runs the hand-written
adjoint kernels (fwime_gradient_backward: the Born adjoint B* r and the
tomographic adjoint T* r, recomputing the source-side wavefields segment by
segment from those checkpoints) and scales the result by the incoming
gradient.  When v does not require a gradient only the objective is computed
and nothing is kept.  p~ is held fixed (the variable-projection gradient, whose
chain through p~_opt vanishes at the optimum), so no gradient flows to p~.
"""
from __future__ import annotations

import torch


class FwimeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, context, w, pt, dobs, eps):
        vd = v.detach().contiguous()
        if ctx.needs_input_grad[0]:
            J = context.gradient_forward(vd, w, pt, dobs, eps=eps)
            # the adjoint half needs the same v, w and p~ memory that the forward half saw
            ctx.save_for_backward(vd)
            ctx.context, ctx.w, ctx.pt, ctx.dobs, ctx.eps = context, w, pt, dobs, eps
        else:
            J = context.objective(vd, w, pt, dobs, eps=eps)
        return torch.tensor(J, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, gJ):
        (vd,) = ctx.saved_tensors
        grad = torch.empty_like(vd)
        ctx.context.gradient_backward(vd, ctx.w, ctx.pt, ctx.dobs, grad, eps=ctx.eps)
        return (gJ.reshape(()).to(grad.dtype) * grad, None, None, None, None, None)


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
