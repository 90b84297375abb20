"""torch.autograd.Function over the library's render / render-backward kernels.

The forward renders a ray batch (§III-B "Volume Rendering", Eq. 7) from a
parameter tensor theta; the backward runs the hand-written adjoint kernel
(compositing, MLP and hash-grid scatter) for the upstream gradients of the
colour, depth and opacity, and returns dL/dtheta.  theta is copied into the
object's parameter buffer before each kernel, so any torch tensor holding the
object's parameters (in the layout of include/prenom.h) can be the leaf.
"""

from __future__ import annotations

import torch

from . import PRENOM_STATE_THETA


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, context, obj, batch, opts):
        context.set_state(obj, PRENOM_STATE_THETA, theta.detach().contiguous())
        out = context.render(batch, opts)
        ctx.context = context
        ctx.obj = obj
        ctx.batch = batch
        ctx.opts = opts
        ctx.save_for_backward(theta)
        return out["rgb"], out["depth"], out["acc"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_acc):
        (theta,) = ctx.saved_tensors
        n = ctx.batch["o"].shape[0]
        dev = theta.device
        g_rgb = g_rgb if g_rgb is not None else torch.zeros((n, 3), device=dev)
        g_depth = g_depth if g_depth is not None else torch.zeros(n, device=dev)
        g_acc = g_acc if g_acc is not None else torch.zeros(n, device=dev)
        d_out = torch.cat([g_rgb.reshape(n, 3), g_depth.reshape(n, 1), g_acc.reshape(n, 1)], dim=1)
        d_out = d_out.to(torch.float32).contiguous()
        grad = torch.zeros_like(theta, dtype=torch.float32)
        ctx.context.set_state(ctx.obj, PRENOM_STATE_THETA, theta.detach().contiguous())
        ctx.context.render_backward(ctx.batch, ctx.opts, d_out, grad)
        return grad, None, None, None, None


def render(context, obj: int, theta: torch.Tensor, batch: dict, opts):
    """(rgb [n,3], depth [n], acc [n]) differentiable with respect to theta."""
    return RenderFunction.apply(theta, context, obj, batch, opts)
