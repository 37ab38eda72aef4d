"""torch.autograd.Function over the C-ABI operators.

``CTProject.apply(x, theta, delta, op)`` returns H(theta, delta) x through
``ct_forward``; its backward returns
    dL/dx     = H^T g                (ct_adjoint, the gather transpose)
    dL/dtheta = sum_k J_theta(x_k)^T g_k   (ct_jacT_batch, summed over the batch in the kernel)
    dL/ddelta = sum_k J_delta(x_k)^T g_k   (ct_jacT_batch)
for the incoming gradient g (one image or a batch of images x_k).  Those are the gradient components
[grad_p J]_i = (H_{p_i} u)^T (H u - b) of the appendix lemma on the
Lipschitz gradient when the loss is 1/2 |H u - b|^2.  Everything runs in the
library's kernels; nothing is differentiated by torch itself.
"""
from __future__ import annotations

import torch

from .ct import CTOperator


class CTProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, delta, op: CTOperator):
        y = op.forward(x.contiguous(), theta.detach().contiguous(),
                       None if delta is None else delta.detach().contiguous())
        ctx.op = op
        ctx.has_delta = delta is not None
        ctx.save_for_backward(x, theta, delta if delta is not None else theta.new_empty(0))
        return y

    @staticmethod
    def backward(ctx, gy):
        x, theta, delta = ctx.saved_tensors
        op = ctx.op
        d = delta if ctx.has_delta else None
        gy = gy.contiguous()
        gx = gth = gdl = None
        if ctx.needs_input_grad[0]:
            gx = op.adjoint(gy, theta, d)
        if ctx.needs_input_grad[1] or (ctx.has_delta and ctx.needs_input_grad[2]):
            # one launch over the whole batch; the kernel adds the images' gradients in order
            xs = x.reshape(-1, op.n).contiguous()
            gs = gy.reshape(-1, op.m).contiguous()
            if ctx.has_delta:
                gth, gdl = op.jacT_batch(xs, theta, gs, d, want_delta=True, sum_images=True)
            else:
                gth, gdl = op.jacT_batch(xs, theta, gs, sum_images=True), None
            if not ctx.needs_input_grad[1]:
                gth = None
            if not (ctx.has_delta and ctx.needs_input_grad[2]):
                gdl = None
        return gx, gth, gdl, None


def project(x, theta, op: CTOperator, delta=None):
    """y = H(theta, delta) x, differentiable in x, theta and delta."""
    return CTProject.apply(x, theta, delta, op)


class VarProObjective(torch.autograd.Function):
    """f(theta) of the VarPro reduced problem on a fixed basis (Sec. 4.2).

    The inner reduced solve is not stored: backward recomputes it at the
    saved angles (checkpointing) through ``nlrmm_varpro``, whose gradient is
    J_theta(u)^T (H u - b) at the optimal u = V y (envelope form).
    """

    @staticmethod
    def forward(ctx, theta, op: CTOperator, b, V, lam, u_w=None, eps=1e-3):
        f, _, _ = op.varpro(b, theta.detach().contiguous(), V, lam, u_w, eps, want_grad=False)
        ctx.op, ctx.lam, ctx.eps = op, lam, eps
        ctx.save_for_backward(theta, b, V, u_w if u_w is not None else theta.new_empty(0))
        ctx.has_w = u_w is not None
        return f.reshape(())

    @staticmethod
    def backward(ctx, gf):
        theta, b, V, u_w = ctx.saved_tensors
        _, grad, _ = ctx.op.varpro(b, theta.detach().contiguous(), V, ctx.lam, u_w if ctx.has_w else None, ctx.eps)
        return gf * grad, None, None, None, None, None, None


def varpro_objective(theta, op: CTOperator, b, V, lam, u_w=None, eps=1e-3):
    """Differentiable VarPro reduced objective f(theta)."""
    return VarProObjective.apply(theta, op, b, V, lam, u_w, eps)
