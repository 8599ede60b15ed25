"""PyTorch autograd wrapper of the warp + LNCC loss (forward and all three
adjoints in one libfa call, fa_warp_lncc_adjoint).

    loss = warp_lncc(fixed, moving, u, window=5, cc_eps=1e-5)
    loss.backward()        # fills fixed.grad, moving.grad, u.grad as requested

L = LNCC(I_f, I_m o (id + u)) (reading R-lncc); dL/du is the Gateaux
derivative of section "Jacobian-free Eulerian descent", dL/dI_m the adjoint
of the trilinear warp.  The gradients are computed during the forward call
(they come from the same window sums) and scaled by the incoming gradient in
backward.  CUDA float32 tensors only; there is no CPU path.
"""
from __future__ import annotations

import torch

from . import fa


class WarpLNCC(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fixed, moving, u, window: int = 5, cc_eps: float = 1e-5):
        need = ctx.needs_input_grad
        r = fa.fa_warp_lncc_adjoint(fixed.detach().contiguous(), moving.detach().contiguous(),
                                    u.detach().contiguous(), window, cc_eps,
                                    want_u=bool(need[2]), want_fixed=bool(need[0]),
                                    want_moving=bool(need[1]))
        ctx.save_for_backward(r["dL_dfixed"], r["dL_dmoving"], r["dL_du"])
        return r["loss"]

    @staticmethod
    def backward(ctx, gout):
        dfx, dmv, du = ctx.saved_tensors
        scale = lambda t: None if t is None else gout * t  # noqa: E731
        return scale(dfx), scale(dmv), scale(du), None, None


def warp_lncc(fixed: torch.Tensor, moving: torch.Tensor, u: torch.Tensor, window: int = 5,
              cc_eps: float = 1e-5) -> torch.Tensor:
    """Differentiable LNCC loss of fixed and moving warped by u ([3, D, H, W])."""
    return WarpLNCC.apply(fixed, moving, u, window, cc_eps)
