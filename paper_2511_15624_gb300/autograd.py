"""``torch.autograd.Function`` over the certified bound.

Forward: ``ibp_bound`` on device tensors (obj_lo, obj_hi).  Backward:
``ibp_bound_backward``, the hand-written adjoint of obj_hi with respect to the
box endpoints.  obj_lo is returned as a non-differentiable output (the adjoint
of the lower bound is not provided).
"""
from __future__ import annotations

import torch

from .case import Case


class IBPBoundFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, box_lo: torch.Tensor, box_hi: torch.Tensor, case: Case):
        lo = box_lo.detach().contiguous().to(torch.float64)
        hi = box_hi.detach().contiguous().to(torch.float64)
        obj_lo, obj_hi, _ = case.bound(lo, hi)
        ctx.case = case
        ctx.save_for_backward(lo, hi)
        ctx.mark_non_differentiable(obj_lo)
        return obj_lo, obj_hi

    @staticmethod
    def backward(ctx, grad_obj_lo, grad_obj_hi):
        lo, hi = ctx.saved_tensors
        if grad_obj_hi is None:
            return None, None, None
        g = grad_obj_hi.detach().contiguous().to(torch.float64)
        glo, ghi = ctx.case.backward(lo, hi, g)
        return glo, ghi, None


def ibp_bound(case: Case, box_lo: torch.Tensor, box_hi: torch.Tensor):
    """Differentiable (obj_lo, obj_hi) of every box; gradients flow through obj_hi."""
    return IBPBoundFunction.apply(box_lo, box_hi, case)


__all__ = ["IBPBoundFunction", "ibp_bound"]
