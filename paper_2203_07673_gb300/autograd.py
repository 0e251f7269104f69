"""FusedMM as a differentiable PyTorch op (hand-written adjoint).

``fusedmm(plan, vals, A, B)`` returns FusedMMA(S, A, B) (m x r, float32) and
``fusedmm(plan, vals, A, B, transpose=True)`` returns FusedMMB (n x r), both
from the fused CUDA kernels of libfmm.  Backward calls the library's adjoint
(fmm_fusedmm_bwd / fmm_fusedmm_t_bwd): each gradient is itself an SDDMM- or
SpMM-shaped pass over the same pattern, and the SDDMM values are recomputed
rather than stored.  Gradients flow to ``vals`` (the values of S on the fixed
pattern), ``A`` and ``B``; bfloat16 inputs receive bfloat16 gradients
(computed in float32, rounded once).
"""
from __future__ import annotations

import torch

from . import fmm


class FusedMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, vals, A, B, transpose=False):
        out = (fmm.fusedmm_t if transpose else fmm.fusedmm)(plan, vals, A, B)
        ctx.plan = plan
        ctx.transpose = transpose
        ctx.save_for_backward(vals, A, B)
        return out

    @staticmethod
    def backward(ctx, G):
        vals, A, B = ctx.saved_tensors
        G = G.contiguous()
        if G.dtype != torch.float32:
            G = G.float()
        need = (ctx.needs_input_grad[2], ctx.needs_input_grad[3],
                vals is not None and ctx.needs_input_grad[1])
        if not any(need):
            return None, None, None, None, None
        fn = fmm.fusedmm_t_bwd if ctx.transpose else fmm.fusedmm_bwd
        dA, dB, ds = fn(ctx.plan, vals, A, B, G, need)
        if dA is not None and dA.dtype != A.dtype:
            dA = dA.to(A.dtype)
        if dB is not None and dB.dtype != B.dtype:
            dB = dB.to(B.dtype)
        return None, ds, dA, dB, None


def fusedmm(plan, vals, A, B, transpose: bool = False):
    """Differentiable FusedMMA (or FusedMMB with transpose=True)."""
    return FusedMMFunction.apply(plan, vals, A, B, transpose)
