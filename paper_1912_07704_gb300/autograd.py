"""torch.autograd bindings of the differentiable dedispersion.

* ``Dedisperse.apply(x, w, plan)``: y = sum_c w_c x[c][t + s(c,d)]; the
  backward runs the transpose (adjoint) kernel for x and the weight gradient
  in the same pass.  Only x and w are saved for backward.
* ``DedispersionMSE.apply(x, w, template, plan)``: mean((y - T)^2) reduced
  inside the forward kernel; its backward recomputes y in chunks of DM
  trials, so the DM x time intermediate is never stored whole.

x is float32 [nchans][nsamp] (contiguous rows), w float32 [nchans]; y and
the template use the flat layout of ``Plan.alloc_output``.
"""
from __future__ import annotations

import torch


class Dedisperse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, plan):
        ctx.plan = plan
        ctx.save_for_backward(x, w)
        return plan.f32_forward(x.contiguous(), w.contiguous())

    @staticmethod
    def backward(ctx, gy):
        x, w = ctx.saved_tensors
        gx, gw = ctx.plan.f32_adjoint(x.contiguous(), w.contiguous(), gy.contiguous())
        return gx, gw, None


class DedispersionMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, template, plan):
        ctx.plan = plan
        ctx.save_for_backward(x, w, template)
        loss, _, _ = plan.f32_mse(x.contiguous(), w.contiguous(), template.contiguous())
        return loss

    @staticmethod
    def backward(ctx, gl):
        x, w, template = ctx.saved_tensors
        _, gx, gw = ctx.plan.f32_mse(x.contiguous(), w.contiguous(), template.contiguous(),
                                     grad=True)
        s = gl.to(torch.float32)
        return gx * s, gw * s, None, None
