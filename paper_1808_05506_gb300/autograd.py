"""Differentiable out = D(V) psi for the staggered, Wilson and Brillouin operators.

forward:  out = D psi (dirac_apply)
backward: dL/dpsi = D^+ g (dirac_apply_dagger) and dL/dV = the link force
          (dirac_force; for Brillouin through the transporters W, which the
          backward pass rebuilds from V), both hand-written kernels of the library, with
          PyTorch's convention for real losses of complex tensors
          (grad = dL/dRe + i dL/dIm), so that for L = Re <g, D psi> the
          gradients are exactly D^+ g and F.
"""
from __future__ import annotations

import torch

from . import Dirac


class DiracApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, V, D: Dirac):
        D.set_links(V.detach())
        out = D.apply(psi.detach().to(D.canon_dtype).contiguous())
        ctx.D = D
        ctx.save_for_backward(psi, V)
        return out

    @staticmethod
    def backward(ctx, g):
        D = ctx.D
        psi, V = ctx.saved_tensors
        g = g.to(D.canon_dtype).contiguous()
        # the handle may have been reused with other links since the forward pass
        D.set_links(V.detach())
        gpsi = gV = None
        if ctx.needs_input_grad[0]:
            gpsi = D.apply_dagger(g).to(psi.dtype)
        if ctx.needs_input_grad[1]:
            gV = D.force(psi.detach().to(D.canon_dtype).contiguous(), g).to(V.dtype)
        return gpsi, gV, None


def dirac_apply(D: Dirac, psi: torch.Tensor, V: torch.Tensor) -> torch.Tensor:
    """out = D(V) psi, differentiable in psi and V."""
    return DiracApply.apply(psi, V, D)
