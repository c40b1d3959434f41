"""torch.autograd.Function around libqtp's forward and hand-written backward.

Forward: C = A * B (Algorithm 5.1).  Backward, for a real loss with each
quaternion entry taken as four reals: dA = dC * B^H, dB = A^H * dC (tensor
conjugate transpose, Kilmer-Martin convention).  When a gradient is needed the
forward runs qtp_forward_saving, which keeps the spectra of A and B in a buffer
of this call, and the backward qtp_backward_saved, which reuses them (only dC
is transformed again).  Both run in libqtp's CUDA kernels; torch only supplies
memory and streams.
"""
from __future__ import annotations

import torch

from . import qtp


class TProduct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, precision="bf16x3"):
        A = A.contiguous()
        B = B.contiguous()
        _, m, n, p, _ = A.shape
        s = B.shape[2]
        plan = qtp.plan_for(m, n, s, p, precision)
        ctx.plan = plan
        if not (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            ctx.spectra = None
            return plan.forward(A, B)
        C, ctx.spectra = plan.forward_saving(A, B)
        return C

    @staticmethod
    def backward(ctx, dC):
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_a or need_b) or ctx.spectra is None:
            return None, None, None
        dA, dB = ctx.plan.backward_saved(dC.contiguous(), ctx.spectra, need_dA=need_a, need_dB=need_b)
        return dA, dB, None


def tprod(A, B, precision="bf16x3"):
    """Differentiable T-product of quaternion tensors in plane layout."""
    return TProduct.apply(A, B, precision)
