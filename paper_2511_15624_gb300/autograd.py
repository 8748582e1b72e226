"""``torch.autograd.Function`` over the certified bound.

Forward: ``ibp_bound`` on device tensors, returning (obj_lo, obj_hi).  With a
``rating`` tensor the case's line ratings (base and contingency together) are
first replaced by it (``ibp_case_set_ratings``), so the bound is a function of
the box endpoints and of the ratings.  Backward: the hand-written adjoints --
``ibp_bound_backward`` for obj_hi and ``ibp_bound_backward_lo`` for obj_lo --
with respect to the box endpoints and the ratings; each is taken with the
active set of its own forward pass and is valid away from kinks.
"""
from __future__ import annotations

from typing import Optional

import torch

from .case import Case


class IBPBoundFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, box_lo: torch.Tensor, box_hi: torch.Tensor, rating: Optional[torch.Tensor],
                case: Case):
        lo = box_lo.detach().contiguous().to(torch.float64)
        hi = box_hi.detach().contiguous().to(torch.float64)
        if rating is not None:
            case.set_ratings(rating.detach().contiguous().to(torch.float64))
        obj_lo, obj_hi, _ = case.bound(lo, hi)
        ctx.case = case
        ctx.has_rating = rating is not None
        ctx.save_for_backward(lo, hi, None if rating is None else rating.detach())
        return obj_lo, obj_hi

    @staticmethod
    def backward(ctx, grad_obj_lo, grad_obj_hi):
        lo, hi, rating = ctx.saved_tensors
        want_r = ctx.has_rating and ctx.needs_input_grad[2]
        if rating is not None:
            # the ratings this forward pass used (another call may have changed them)
            ctx.case.set_ratings(rating.contiguous().to(torch.float64))
        glo = torch.zeros_like(lo)
        ghi = torch.zeros_like(hi)
        grat = torch.zeros(lo.shape[0], ctx.case.n_line, dtype=torch.float64, device=lo.device) \
            if want_r else None
        for side, g in (("hi", grad_obj_hi), ("lo", grad_obj_lo)):
            if g is None:
                continue
            g = g.detach().contiguous().to(torch.float64)
            out = ctx.case.backward(lo, hi, g, want_rating=want_r, side=side)
            glo += out[0]
            ghi += out[1]
            if want_r:
                grat += out[2]
        return glo, ghi, (grat.sum(dim=0) if want_r else None), None


def ibp_bound(case: Case, box_lo: torch.Tensor, box_hi: torch.Tensor,
              rating: Optional[torch.Tensor] = None):
    """Differentiable (obj_lo, obj_hi) of every box; gradients flow to the box
    endpoints and, when given, to the line ratings."""
    return IBPBoundFunction.apply(box_lo, box_hi, rating, case)


__all__ = ["IBPBoundFunction", "ibp_bound"]
