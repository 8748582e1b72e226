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
        # an end the loss does not use gets no gradient (None): its adjoint pass is skipped
        ctx.set_materialize_grads(False)
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


class IBPBoundMultiFunction(torch.autograd.Function):
    """Many cases of uneven size: forward in one persistent launch
    (``ibp_bound_multi``), backward through ``ibp_bound_multi_backward``
    (one launch per backward pass over all cases).  Inputs after ``cases``:
    box_lo_0, box_hi_0, box_lo_1, box_hi_1, ...; outputs: obj_lo_0,
    obj_hi_0, obj_lo_1, obj_hi_1, ...  Like every call on device tensors,
    device-side errors surface at ``Case.sync()`` of the case concerned."""

    @staticmethod
    def forward(ctx, cases, *boxes):
        from .case import bound_multi
        los = [b.detach().contiguous().to(torch.float64) for b in boxes[0::2]]
        his = [b.detach().contiguous().to(torch.float64) for b in boxes[1::2]]
        outs = bound_multi(list(cases), los, his)
        ctx.set_materialize_grads(False)
        ctx.cases = list(cases)
        ctx.save_for_backward(*[t for pair in zip(los, his) for t in pair])
        return tuple(t for o in outs for t in (o[0], o[1]))

    @staticmethod
    def backward(ctx, *grads):
        from .case import bound_multi_backward
        saved = ctx.saved_tensors
        los, his = list(saved[0::2]), list(saved[1::2])
        g_lo = [torch.zeros_like(lo) for lo in los]
        g_hi = [torch.zeros_like(hi) for hi in his]
        for side, gs in (("hi", grads[1::2]), ("lo", grads[0::2])):
            if all(g is None for g in gs):
                continue
            gobj = [torch.zeros(lo.shape[0], dtype=torch.float64, device=lo.device) if g is None
                    else g.detach().to(torch.float64) for g, lo in zip(gs, los)]
            for i, (a, b, _) in enumerate(bound_multi_backward(ctx.cases, los, his, gobj, side=side)):
                g_lo[i] += a
                g_hi[i] += b
        return (None,) + tuple(t for pair in zip(g_lo, g_hi) for t in pair)


def ibp_bound_multi(cases, box_lo, box_hi):
    """Differentiable [(obj_lo, obj_hi)] of many cases, one persistent launch
    forward and one batched adjoint backward."""
    flat = [t for pair in zip(box_lo, box_hi) for t in pair]
    out = IBPBoundMultiFunction.apply(tuple(cases), *flat)
    return [(out[2 * i], out[2 * i + 1]) for i in range(len(cases))]


def ibp_bound(case: Case, box_lo: torch.Tensor, box_hi: torch.Tensor,
              rating: Optional[torch.Tensor] = None):
    """Differentiable (obj_lo, obj_hi) of every box; gradients flow to the box
    endpoints and, when given, to the line ratings."""
    return IBPBoundFunction.apply(box_lo, box_hi, rating, case)


__all__ = ["IBPBoundFunction", "IBPBoundMultiFunction", "ibp_bound", "ibp_bound_multi"]
