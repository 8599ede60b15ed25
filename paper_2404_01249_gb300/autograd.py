"""PyTorch autograd wrapper of the warp + LNCC loss (libfa's
fa_warp_lncc_adjoint).

    loss = warp_lncc(fixed, moving, u, window=5, cc_eps=1e-5)
    loss.backward()        # fills fixed.grad, moving.grad, u.grad as requested

L = LNCC(I_f, I_m o (id + u)) (reading R-lncc); dL/du is the Gateaux
derivative of section "Jacobian-free Eulerian descent", dL/dI_m the adjoint
of the trilinear warp (template building).  forward evaluates the loss alone
(warp and the forward window sums; no gradient volume is formed) and keeps
the three inputs; backward recomputes the warp and the window sums and runs
the adjoint for exactly the inputs that need a gradient, so nothing of the
size of a volume lives between the two passes beyond the inputs themselves.
CUDA float32 tensors only; there is no CPU path.
"""
from __future__ import annotations

import torch

from . import fa


class WarpLNCC(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fixed, moving, u, window: int = 5, cc_eps: float = 1e-5):
        fixed, moving, u = fixed.detach().contiguous(), moving.detach().contiguous(), \
            u.detach().contiguous()
        r = fa.fa_warp_lncc_adjoint(fixed, moving, u, window, cc_eps, want_u=False,
                                    want_fixed=False, want_moving=False)
        ctx.save_for_backward(fixed, moving, u)
        ctx.window, ctx.cc_eps = window, cc_eps
        return r["loss"]

    @staticmethod
    def backward(ctx, gout):
        fixed, moving, u = ctx.saved_tensors
        need = ctx.needs_input_grad
        if not (need[0] or need[1] or need[2]):
            return None, None, None, None, None
        r = fa.fa_warp_lncc_adjoint(fixed, moving, u, ctx.window, ctx.cc_eps,
                                    want_u=bool(need[2]), want_fixed=bool(need[0]),
                                    want_moving=bool(need[1]))
        scale = lambda t: None if t is None else gout * t  # noqa: E731
        return scale(r["dL_dfixed"]), scale(r["dL_dmoving"]), scale(r["dL_du"]), None, None


def warp_lncc(fixed: torch.Tensor, moving: torch.Tensor, u: torch.Tensor, window: int = 5,
              cc_eps: float = 1e-5) -> torch.Tensor:
    """Differentiable LNCC loss of fixed and moving warped by u ([3, D, H, W])."""
    return WarpLNCC.apply(fixed, moving, u, window, cc_eps)
