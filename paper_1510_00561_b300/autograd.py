"""Differentiable contourlet transform for gradient-based tuning of subband
thresholds (rate-distortion tuning of the codec's thresholding step, §3.5).

Each Function's forward runs a library kernel and its backward runs the
hand-written adjoint kernel of the same map (no autograd tape through the
transform):

    ct_forward(x)          A x            backward  A^T g   (cvc_ct_forward_adjoint)
    ct_inverse(c)          S c            backward  S^T g   (cvc_ct_inverse_adjoint)
    soft_threshold(c, T)   per-subband    backward  cvc_ct_soft_threshold_backward

ThresholdedReconstruction chains them: x -> S(soft_T(A x)), with a learnable
threshold per directional subband.
"""
import torch

from .codec import CtPlan


class _CtForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.forward_adjoint(g.contiguous()), None


class _CtInverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, plan):
        ctx.plan = plan
        return plan.inverse(c.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.inverse_adjoint(g.contiguous()), None


class _SoftThreshold(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, T, plan):
        c = c.contiguous()
        T = T.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(c, T)
        return plan.soft_threshold(c, T)

    @staticmethod
    def backward(ctx, g):
        c, T = ctx.saved_tensors
        gc, gT = ctx.plan.soft_threshold_backward(c, T, g.contiguous())
        return gc, gT, None


def ct_forward(x, plan):
    """A x for planes x of shape (plan.batch, plan.h, plan.w)."""
    return _CtForward.apply(x, plan)


def ct_inverse(c, plan):
    """S c for coefficients c of shape (plan.batch, plan.total)."""
    return _CtInverse.apply(c, plan)


def soft_threshold(c, T, plan):
    """sign(c) max(|c| - T[s], 0) in each directional subband s; lowpass unchanged."""
    return _SoftThreshold.apply(c, T, plan)


class ThresholdedReconstruction(torch.nn.Module):
    """x -> S(soft_T(A x)) with one learnable threshold per directional subband."""

    def __init__(self, height, width, levels, dirs_log2, batch, t_init=4.0, device="cuda"):
        super().__init__()
        self.plan = CtPlan(height, width, levels, dirs_log2, batch)
        self.T = torch.nn.Parameter(torch.full((self.plan.subbands,), float(t_init), device=device))

    def forward(self, x):
        return ct_inverse(soft_threshold(ct_forward(x, self.plan), self.T, self.plan), self.plan)
