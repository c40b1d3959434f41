"""torch.autograd.Function around libqtp's forward and hand-written backward.

Forward: C = A * B (Algorithm 5.1).  Backward, for a real loss with each
quaternion entry taken as four reals: dA = dC * B^H, dB = A^H * dC (tensor
conjugate transpose, Kilmer-Martin convention), computed by qtp_backward.
Both run in libqtp's CUDA kernels; torch only supplies memory and streams.
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
        ctx.save_for_backward(A, B)
        ctx.plan = plan
        return plan.forward(A, B)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_a or need_b):
            return None, None, None
        dA, dB = ctx.plan.backward(dC.contiguous(), A, B, need_dA=need_a, need_dB=need_b)
        return dA, dB, None


def tprod(A, B, precision="bf16x3"):
    """Differentiable T-product of quaternion tensors in plane layout."""
    return TProduct.apply(A, B, precision)
