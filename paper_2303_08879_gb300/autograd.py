"""torch.autograd.Function wrappers around the C ABI.

The forward leaves the walk's amplitudes in a workspace that the backward
reuses, so one forward + backward costs one forward walk plus one reverse
walk (Sec. 2.5's gradients, computed in reverse mode instead of carrying the
1 + D + D^2 forward-mode tangents).
"""
from __future__ import annotations

import torch

from . import fockdiag as fd


class FockDiagProbs(torch.autograd.Function):
    """probs[B, *cutoffs] = p(n) of Algorithm 1 for a batch of circuits."""

    @staticmethod
    def forward(ctx, A, b, c, cutoffs, flags=0):
        probs, ws = fd.fock_diag_probs_batched(A.contiguous(), b.contiguous(), c.contiguous(),
                                               cutoffs, flags=flags)
        ctx.save_for_backward(A, b, c)
        ctx.ws = ws
        ctx.cutoffs = tuple(cutoffs)
        ctx.flags = flags
        return probs

    @staticmethod
    def backward(ctx, grad_probs):
        A, b, c = ctx.saved_tensors
        gA, gb, gc = fd.fock_diag_probs_vjp_batched(A.contiguous(), b.contiguous(), c.contiguous(),
                                                    ctx.cutoffs, grad_probs.contiguous(), ctx.ws,
                                                    flags=ctx.flags)
        ctx.ws = None
        return gA, gb, gc, None, None


def diag_probs(A, b, c, cutoffs, flags=0):
    """Differentiable p(n): A [B, D, D], b [B, D], c [B] (complex128, CUDA)."""
    return FockDiagProbs.apply(A, b, c, tuple(cutoffs), flags)
