"""Python-side handle of an IBP case (a thin wrapper of the C ABI).

``Case`` owns one ``ibp_case``; ``Case.bound`` and ``Case.backward`` marshal
numpy (host) or torch CUDA (device) arrays into ``ibp_bound`` and
``ibp_bound_backward``.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _abi


class Case:
    """A network, its devices, prices and contingency list, built on one GPU.

    ``network`` is any object with the attributes of ``gen.Case`` (n_bus, slack,
    line_from, line_to, reactance, rating, gen_bus, gen_nseg, gen_slope,
    gen_bkpt, load_bus, load_nseg, load_slope, load_bkpt, zeta_inj, zeta_f,
    ctg_line and optionally rating_ctg).
    """

    def __init__(self, network, device: int = 0):
        n = network
        self.n_bus = int(n.n_bus)
        self.n_line = int(len(n.line_from))
        self.n_gen = int(len(n.gen_bus))
        self.n_load = int(len(n.load_bus))
        self.n_dev = self.n_gen + self.n_load
        self.n_ctg = int(len(n.ctg_line))
        self.device = device
        self._h = None
        self._h = _abi.ibp_case_create(
            n.n_bus, n.slack, n.line_from, n.line_to, n.reactance, n.rating,
            getattr(n, "rating_ctg", None), n.gen_bus, n.gen_nseg, n.gen_slope, n.gen_bkpt,
            n.load_bus, n.load_nseg, n.load_slope, n.load_bkpt, n.zeta_inj, n.zeta_f,
            n.ctg_line, device)

    @property
    def handle(self) -> int:
        return self._h

    def close(self):
        if self._h is not None:
            _abi.ibp_case_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> _abi.CaseInfo:
        return _abi.ibp_case_info(self._h)

    # ------------------------------------------------------------ forward
    def bound(self, lo, hi, flows: bool = False, stream=None):
        """Certified IBP bound over each box.

        Host (numpy) boxes: returns numpy ``(obj_lo, obj_hi, obj_err)`` with
        ``obj_err[:, 0]`` bounding the error of obj_hi and ``obj_err[:, 1]`` that
        of obj_lo, and, if
        ``flows``, ``(flow_lo, flow_hi)`` of shape [n_box, n_ctg, n_line].
        CUDA tensors: the same as torch tensors, enqueued on ``stream`` (default:
        torch's current stream) without synchronising.
        """
        if _abi._is_cuda_tensor(lo):
            import torch
            lo = lo.contiguous().to(torch.float64)
            hi = hi.contiguous().to(torch.float64)
            nb = int(lo.shape[0]) if lo.dim() == 2 else 1
            out = torch.empty((2, nb), dtype=torch.float64, device=lo.device)
            err = torch.empty((nb, 2), dtype=torch.float64, device=lo.device)
            fl = fh = None
            if flows:
                fl = torch.empty((nb, self.n_ctg, self.n_line), dtype=torch.float32, device=lo.device)
                fh = torch.empty_like(fl)
            s = stream if stream is not None else torch.cuda.current_stream(lo.device).cuda_stream
            _abi.ibp_bound(self._h, nb, lo, hi, out[0], out[1], err, fl, fh, ptr_mode=1,
                           stream=s)
            res = (out[0], out[1], err)
            return res + ((fl, fh) if flows else ())
        lo = np.ascontiguousarray(np.atleast_2d(lo), np.float64)
        hi = np.ascontiguousarray(np.atleast_2d(hi), np.float64)
        if lo.shape != hi.shape or lo.shape[1] != self.n_dev:
            raise ValueError(f"boxes must be [n_box, {self.n_dev}]")
        nb = lo.shape[0]
        olo, ohi, oerr = np.empty(nb), np.empty(nb), np.empty((nb, 2))
        fl = fh = None
        if flows:
            fl = np.empty((nb, self.n_ctg, self.n_line), np.float32)
            fh = np.empty_like(fl)
        _abi.ibp_bound(self._h, nb, lo, hi, olo, ohi, oerr, fl, fh, ptr_mode=0, stream=None)
        return (olo, ohi, oerr) + ((fl, fh) if flows else ())

    def bound_paper(self, lo, hi, stream=None):
        """The objective interval with the paper's two-part contingency
        intervals (looser than ``bound``, O(n_ctg * n_line)); same argument
        and return conventions as ``bound`` without flows."""
        if _abi._is_cuda_tensor(lo):
            import torch
            lo = lo.contiguous().to(torch.float64)
            hi = hi.contiguous().to(torch.float64)
            nb = int(lo.shape[0]) if lo.dim() == 2 else 1
            out = torch.empty((2, nb), dtype=torch.float64, device=lo.device)
            err = torch.empty((nb, 2), dtype=torch.float64, device=lo.device)
            s = stream if stream is not None else torch.cuda.current_stream(lo.device).cuda_stream
            _abi.ibp_bound_paper(self._h, nb, lo, hi, out[0], out[1], err, ptr_mode=1, stream=s)
            return out[0], out[1], err
        lo = np.ascontiguousarray(np.atleast_2d(lo), np.float64)
        hi = np.ascontiguousarray(np.atleast_2d(hi), np.float64)
        if lo.shape != hi.shape or lo.shape[1] != self.n_dev:
            raise ValueError(f"boxes must be [n_box, {self.n_dev}]")
        nb = lo.shape[0]
        olo, ohi, oerr = np.empty(nb), np.empty(nb), np.empty((nb, 2))
        _abi.ibp_bound_paper(self._h, nb, lo, hi, olo, ohi, oerr, ptr_mode=0, stream=None)
        return olo, ohi, oerr

    # ------------------------------------------------------------ adjoint
    def backward(self, lo, hi, grad_obj_hi, want_rating: bool = False, stream=None, side: str = "hi"):
        """d loss / d box_lo, d box_hi (and d loss / d rating, base and
        contingency ratings moving together) of obj_hi (side "hi",
        ``ibp_bound_backward``) or of obj_lo (side "lo",
        ``ibp_bound_backward_lo``); grad_obj_hi is d loss / d obj of that side."""
        fn = _abi.ibp_bound_backward if side == "hi" else _abi.ibp_bound_backward_lo
        if _abi._is_cuda_tensor(lo):
            import torch
            nb = int(lo.shape[0])
            g = grad_obj_hi.contiguous().to(torch.float64)
            glo = torch.empty((nb, self.n_dev), dtype=torch.float64, device=lo.device)
            ghi = torch.empty_like(glo)
            gr = torch.empty((nb, self.n_line), dtype=torch.float64, device=lo.device) if want_rating else None
            s = stream if stream is not None else torch.cuda.current_stream(lo.device).cuda_stream
            fn(self._h, nb, lo.contiguous(), hi.contiguous(), g, glo, ghi, gr, ptr_mode=1, stream=s)
            return (glo, ghi) + ((gr,) if want_rating else ())
        lo = np.ascontiguousarray(np.atleast_2d(lo), np.float64)
        hi = np.ascontiguousarray(np.atleast_2d(hi), np.float64)
        nb = lo.shape[0]
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(grad_obj_hi, np.float64), (nb,)))
        glo = np.empty((nb, self.n_dev))
        ghi = np.empty((nb, self.n_dev))
        gr = np.empty((nb, self.n_line)) if want_rating else None
        fn(self._h, nb, lo, hi, g, glo, ghi, gr, ptr_mode=0, stream=None)
        return (glo, ghi) + ((gr,) if want_rating else ())

    def bound_linear(self, lo, hi, n_iter: int = 20000, primal_weight: float = 0.01, stream=None,
                     warm: bool = False, first: int = 0):
        """Linear (CROWN-style) relaxation bound with optimised slopes
        (``ibp_bound_linear``): returns (obj_hi, obj_err, x_point) -- the
        certified upper bound of max f, its rounding bound and the averaged
        primal point -- as numpy arrays for numpy boxes, CUDA tensors for CUDA
        boxes (enqueued on the stream).  warm=True continues the held state of
        boxes [first, first + n_box).  The start weight 0.01 balances the
        preconditioned primal and dual steps on the synthetic networks (the
        restarts adapt it)."""
        warm = (1 + int(first)) if warm else 0
        if _abi._is_cuda_tensor(lo):
            import torch
            lo = lo.contiguous().to(torch.float64)
            hi = hi.contiguous().to(torch.float64)
            nb = int(lo.shape[0])
            ub = torch.empty(nb, dtype=torch.float64, device=lo.device)
            err = torch.empty_like(ub)
            xp = torch.empty_like(lo)
            s = stream if stream is not None else torch.cuda.current_stream(lo.device).cuda_stream
            _abi.ibp_bound_linear(self._h, nb, lo, hi, n_iter, primal_weight, ub, err, xp, ptr_mode=1,
                                  stream=s, warm=warm)
            return ub, err, xp
        lo = np.ascontiguousarray(np.atleast_2d(lo), np.float64)
        hi = np.ascontiguousarray(np.atleast_2d(hi), np.float64)
        nb = lo.shape[0]
        ub, err, xp = np.empty(nb), np.empty(nb), np.empty_like(lo)
        _abi.ibp_bound_linear(self._h, nb, lo, hi, n_iter, primal_weight, ub, err, xp, ptr_mode=0,
                              warm=warm)
        return ub, err, xp

    def linear_inherit(self, parent):
        """Box j of the next warm ``bound_linear`` continues from box parent[j]."""
        _abi.ibp_case_linear_inherit(self._h, parent)

    def linear_slopes(self, n_box: int = 1):
        """(a_ctg, a_base, a_inj) of the last ``bound_linear`` call."""
        return _abi.ibp_case_linear_slopes(self._h, n_box, self.n_ctg, self.n_line)

    def set_ratings(self, rating, rating_ctg=None, stream=None):
        """Replace the line ratings (numpy: synchronous; CUDA tensor: enqueued
        on the stream).  rating_ctg None: contingency ratings = rating."""
        if _abi._is_cuda_tensor(rating):
            import torch
            r = rating.detach().contiguous().to(torch.float64)
            rc = None if rating_ctg is None else rating_ctg.detach().contiguous().to(torch.float64)
            s = stream if stream is not None else torch.cuda.current_stream(r.device).cuda_stream
            _abi.ibp_case_set_ratings(self._h, r, rc, ptr_mode=1, stream=s)
            return
        r = np.ascontiguousarray(rating, np.float64)
        rc = None if rating_ctg is None else np.ascontiguousarray(rating_ctg, np.float64)
        if r.shape != (self.n_line,):
            raise ValueError(f"rating must have shape [{self.n_line}]")
        _abi.ibp_case_set_ratings(self._h, r, rc, ptr_mode=0, stream=None)

    def sync(self):
        _abi.ibp_case_sync(self._h)

    def set_variant(self, variant: int):
        _abi.ibp_case_set_variant(self._h, variant)

    def set_screen(self, enable: bool):
        """Paper-mode line screen ahead of the contingency kernel (default on)."""
        _abi.ibp_case_set_screen(self._h, enable)

    def set_reduction(self, enable: bool):
        """Exact network reduction of the contingency pass (default on)."""
        _abi.ibp_case_set_reduction(self._h, enable)

    def set_refine(self, enable: bool):
        """FP64 refinement of the terms that can reach obj_hi (default on)."""
        _abi.ibp_case_set_refine(self._h, enable)

    def reduction(self):
        """(class of each active bus column or -1 for the slack's class,
        bridge flag of each line)."""
        info = self.info()
        return _abi.ibp_case_reduction(self._h, info.n_active, self.n_line)

    def last_live(self):
        """(count, ascending indices) of the lines the screen kept in the last
        bound, or (-1, None) when that call did not screen."""
        return _abi.ibp_case_last_live(self._h, self.n_line)

    def set_timing(self, enable: bool):
        _abi.ibp_case_set_timing(self._h, enable)

    def last_timing(self):
        return _abi.ibp_case_last_timing(self._h)


def dry_run_case(network) -> "Case":
    """A case created without a device: validates inputs only (host tests)."""
    return Case(network, device=-1)


def algorithmic_flop(n_ctg: int, n_line: int, n_active: int, n_box: int) -> float:
    """Flops of the contingency kernel counted as FMAs x 2: one FMA forms each
    |H_k| entry and one accumulates it per box, n_c n_l n_a (1 + B) FMAs."""
    return 2.0 * n_ctg * n_line * n_active * (1 + n_box)


__all__ = ["Case", "dry_run_case", "algorithmic_flop", "bound_multi"]
_ = Optional


def bound_multi(cases, box_lo, box_hi, stream=None):
    """Bounds of many cases (networks of uneven size) in one persistent launch
    of the contingency kernel.  ``box_lo[i]``, ``box_hi[i]`` are CUDA tensors
    [n_box_i, n_dev_i]; returns a list of (obj_lo, obj_hi, obj_err) per case,
    enqueued on ``stream`` (default: torch's current stream).  The first call
    with a given set of cases and box counts builds and uploads the work plan;
    later calls only enqueue kernels and can be captured in a CUDA graph."""
    import torch
    outs = []
    los, his = [], []
    for c, lo, hi in zip(cases, box_lo, box_hi):
        lo = lo.contiguous().to(torch.float64)
        hi = hi.contiguous().to(torch.float64)
        los.append(lo)
        his.append(hi)
        nb = int(lo.shape[0])
        outs.append((torch.empty(nb, dtype=torch.float64, device=lo.device),
                     torch.empty(nb, dtype=torch.float64, device=lo.device),
                     torch.empty((nb, 2), dtype=torch.float64, device=lo.device)))
    dev = los[0].device
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    _abi.ibp_bound_multi([c.handle for c in cases], [int(x.shape[0]) for x in los], los, his,
                         [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs], stream=s)
    return outs


def bound_multi_backward(cases, box_lo, box_hi, grad_obj, side: str = "hi", want_rating: bool = False,
                         stream=None):
    """Adjoint of many cases' bounds (``ibp_bound_multi_backward``): the
    forward pass in one persistent launch over all cases, then one launch per
    backward pass over every (case, box).  ``grad_obj[i]`` [n_box_i] is
    d loss / d obj_hi (side "hi") or d loss / d obj_lo (side "lo").  Returns a
    list of (grad_lo, grad_hi, grad_rating or None) per case, CUDA tensors
    enqueued on ``stream``."""
    import torch
    if side not in ("hi", "lo"):
        raise ValueError("side must be 'hi' or 'lo'")
    los = [lo.contiguous().to(torch.float64) for lo in box_lo]
    his = [hi.contiguous().to(torch.float64) for hi in box_hi]
    gs = [g.contiguous().to(torch.float64) for g in grad_obj]
    glo = [torch.empty_like(lo) for lo in los]
    ghi = [torch.empty_like(hi) for hi in his]
    grat = [torch.empty(lo.shape[0], c.n_line, dtype=torch.float64, device=lo.device)
            for c, lo in zip(cases, los)] if want_rating else None
    s = stream if stream is not None else torch.cuda.current_stream(los[0].device).cuda_stream
    _abi.ibp_bound_multi_backward([c.handle for c in cases], [int(x.shape[0]) for x in los], los, his, gs,
                                  glo, ghi, grat, side=0 if side == "hi" else 1, stream=s)
    return [(glo[i], ghi[i], None if grat is None else grat[i]) for i in range(len(cases))]
