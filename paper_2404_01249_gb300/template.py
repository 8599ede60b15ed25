"""Template (atlas) gradient over many subjects, optionally across ranks.

For a template T and subjects S_i with displacements u_i (from registering
each subject), the loss of subject i is L_i = LNCC(S_i, T o (id + u_i)): the
template plays the moving image, warped into every subject's space.  The
template gradient is the mean over all subjects of dL_i/dT; with
torch.distributed initialised it is summed over every rank's subjects with
one all-reduce (sum), then divided by the total subject count, so every
rank gets the same gradient.  The paper builds atlases by repeated template
refinement from many registrations (section "FireANTs facilitates scalable
atlas generation"); this module provides the gradient such a refinement
step uses.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import torch
import torch.distributed as dist


def _cuda_grad(template, subject, u, window, cc_eps):
    from . import fa
    r = fa.fa_warp_lncc_adjoint(subject, template, u, window, cc_eps, want_u=False,
                                want_fixed=False, want_moving=True)
    return r["loss"], r["dL_dmoving"]


def template_gradient(template: torch.Tensor, subjects: Sequence[torch.Tensor],
                      displacements: Sequence[torch.Tensor], window: int = 5,
                      cc_eps: float = 1e-5, group=None,
                      grad_fn: Optional[Callable] = None):
    """Returns (mean loss, mean dL/dT) over the subjects of all ranks.

    grad_fn(template, subject, u, window, cc_eps) -> (loss, dL/dT) computes
    one subject's term; the default runs fa_warp_lncc_adjoint on the GPU."""
    if len(subjects) != len(displacements):
        raise ValueError("one displacement per subject")
    fn = grad_fn or _cuda_grad
    total = torch.zeros_like(template)
    loss = torch.zeros((), dtype=template.dtype, device=template.device)
    for s, u in zip(subjects, displacements):
        li, gi = fn(template, s, u, window, cc_eps)
        total += gi
        loss += li
    count = torch.tensor([float(len(subjects))], dtype=template.dtype, device=template.device)
    if dist.is_available() and dist.is_initialized():
        packed = torch.cat([total.reshape(-1), loss.reshape(1), count])
        dist.all_reduce(packed, op=dist.ReduceOp.SUM, group=group)
        total = packed[:-2].reshape(template.shape)
        loss, count = packed[-2], packed[-1:]
    n = float(count.item())
    if n == 0:
        raise ValueError("no subjects on any rank")
    return loss / n, total / n
