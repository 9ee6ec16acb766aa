"""torch.autograd.Function over the libbez forward and adjoint kernels.

    pts = BezierCurve.apply(ctrl, t)            # integral Bezier curves
    pts = BezierCurve.apply(ctrl, t, weights)   # rational Bezier curves

ctrl [n][d+1][dim] and t ([n_t] shared or [n][n_t] per curve) are CUDA FP32
tensors; gradients flow to ctrl, t and weights.  The forward pass is
bez_eval (de Casteljau) or, for rational curves, bez_eval_nurbs on the single
span of a clamped knot vector with d+1 control points; the backward pass is
bez_eval_backward.  Both run entirely in libbez's kernels.
"""
import torch

from . import bez


class BezierCurve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ctrl, t, weights=None):
        ctrl = ctrl.contiguous()
        t = t.contiguous()
        mode = bez.TMode.SHARED if t.ndim == 1 else bez.TMode.PER_CURVE
        if weights is None:
            out = bez.bez_eval(ctrl, t, variant=bez.Variant.DECASTELJAU, t_mode=mode)
        else:
            weights = weights.contiguous()
            out = bez.bez_eval_nurbs(ctrl, weights, ctrl.shape[1] - 1, t, t_mode=mode)
        ctx.save_for_backward(ctrl, t, weights)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        ctrl, t, weights = ctx.saved_tensors
        gc, gw, gt = bez.bez_eval_backward(ctrl, t, grad_out.contiguous(), weights=weights,
                                           need_ctrl=ctx.needs_input_grad[0], need_t=ctx.needs_input_grad[1],
                                           need_weights=weights is not None and ctx.needs_input_grad[2])
        return gc, gt, gw


def bezier_curve(ctrl, t, weights=None):
    return BezierCurve.apply(ctrl, t, weights)
