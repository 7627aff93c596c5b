"""torch.autograd.Function over the hand-written forward model and adjoint.

`simulate(ctx, O, P, pos)` returns the far-field intensities I [B, N, N]
(arXiv 2505.14372 §3).  Its backward is the library's vector-Jacobian
product (§3.2): the entry waves of every slice are recomputed from O, P and
pos inside the adjoint (nothing but the inputs is saved), and the gradients
follow torch's convention for complex leaves (dL/dRe z + i dL/dIm z).
Any real loss written in torch on I can sit on top.
"""
from __future__ import annotations

import torch

from .api import Context


class PtychoFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, O, P, pos, ctx: Context):
        fctx.ptycho = ctx
        fctx.save_for_backward(O, P, pos)
        return ctx.forward(O.detach().contiguous(), P.detach().contiguous(), pos.detach().contiguous())

    @staticmethod
    def backward(fctx, gI):
        O, P, pos = fctx.saved_tensors
        gO, gP = fctx.ptycho.vjp(O.detach().contiguous(), P.detach().contiguous(), pos.detach().contiguous(),
                                 gI.contiguous().to(torch.float32))
        return (gO if fctx.needs_input_grad[0] else None,
                gP if fctx.needs_input_grad[1] else None, None, None)


def simulate(ctx: Context, O: torch.Tensor, P: torch.Tensor, pos: torch.Tensor) -> torch.Tensor:
    return PtychoFn.apply(O, P, pos, ctx)
