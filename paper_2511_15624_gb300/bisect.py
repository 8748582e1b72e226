"""Gradient-guided input-box bisection on top of the certified bound.

The paper bounds max f over the whole input box with one IBP pass and names
branch-and-bound over the input domain as future work (Sec. I, Sec. V).  This
driver keeps a frontier of leaf boxes that tile the part of the root box that
may still hold the maximiser:

* UB = max over leaves of obj_hi is a certified upper bound of max f over the
  root box (leaves dropped below hold max f <= their obj_hi < LB <= max f);
* LB = max over candidate points x of obj_lo of the zero-width box at x, a
  certified lower bound of f(x) <= max f.  Each leaf carries one candidate
  (its centre at first); every round moves it by a projected sign-gradient
  step inside the leaf, with the gradient of f at x taken from the adjoint of
  the zero-width box (f is concave, so the ascent heads for the maximiser);
* each round bounds every leaf and its centre, takes the adjoint of obj_hi,
  drops leaves with obj_hi < LB, and splits up to ``split_per_round`` leaves
  with the largest obj_hi at the midpoint of the coordinate with the largest
  (|d obj_hi / d lo_i| + |d obj_hi / d hi_i|) * width_i.

``batched=True`` bounds all leaves (and centres) of a round in one call and
takes one adjoint call; ``batched=False`` makes one call per box with the same
split rule.  The frontier (boxes, UB, LB, round) can be saved and reloaded.
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Optional

import numpy as np
import torch

from .case import Case


@dataclasses.dataclass
class RoundRecord:
    round: int
    seconds: float
    ub: float
    lb: float
    gap: float
    n_leaves: int


class Bisection:
    def __init__(self, case: Case, root_lo, root_hi, max_leaves: int = 256,
                 batched: bool = True, device: Optional[torch.device] = None,
                 split_per_round: Optional[int] = None):
        self.case = case
        self.device = device or torch.device("cuda", case.device)
        lo = torch.as_tensor(np.atleast_2d(root_lo), dtype=torch.float64, device=self.device)
        hi = torch.as_tensor(np.atleast_2d(root_hi), dtype=torch.float64, device=self.device)
        self.lo, self.hi = lo.clone(), hi.clone()
        self.max_leaves = int(max_leaves)
        self.split_per_round = int(split_per_round or max(1, self.max_leaves // 16))
        self.batched = bool(batched)
        self.x = 0.5 * (self.lo + self.hi)  # candidate point per leaf
        self.step_frac = 0.25               # ascent step, fraction of the leaf width
        self.ub = float("inf")
        self.lb = -float("inf")
        self.round = 0
        self.history: List[RoundRecord] = []
        self._t0 = None
        self._elapsed = 0.0

    # -------------------------------------------------------------- bounds
    def _bound(self, lo, hi):
        if self.batched:
            obj_lo, obj_hi, _ = self.case.bound(lo, hi)
            return obj_lo, obj_hi
        outs_lo, outs_hi = [], []
        for j in range(lo.shape[0]):
            a, b, _ = self.case.bound(lo[j:j + 1], hi[j:j + 1])
            outs_lo.append(a)
            outs_hi.append(b)
        return torch.cat(outs_lo), torch.cat(outs_hi)

    def _grad(self, lo, hi):
        ones = torch.ones(lo.shape[0], dtype=torch.float64, device=self.device)
        if self.batched:
            return self.case.backward(lo, hi, ones)
        gl, gh = [], []
        for j in range(lo.shape[0]):
            a, b = self.case.backward(lo[j:j + 1], hi[j:j + 1], ones[j:j + 1])
            gl.append(a)
            gh.append(b)
        return torch.cat(gl), torch.cat(gh)

    # -------------------------------------------------------------- rounds
    def step(self) -> RoundRecord:
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        n = self.lo.shape[0]
        both_lo = torch.cat([self.lo, self.x])
        both_hi = torch.cat([self.hi, self.x])
        obj_lo, obj_hi = self._bound(both_lo, both_hi)
        leaf_hi = obj_hi[:n]
        point_lo = obj_lo[n:]
        self.lb = max(self.lb, float(point_lo.max()))
        # projected sign-gradient ascent of every candidate inside its leaf
        gxl, gxh = self._grad(self.x, self.x)
        gx = gxl + gxh
        # components at rounding-noise level count as zero (sign would amplify them)
        gmax = gx.abs().amax(dim=1, keepdim=True)
        gx = torch.where(gx.abs() > 1e-9 * gmax, gx, torch.zeros_like(gx))
        width = self.hi - self.lo
        self.x = torch.minimum(torch.maximum(self.x + self.step_frac * width * torch.sign(gx), self.lo),
                               self.hi)
        self.step_frac *= 0.8
        keep = leaf_hi >= self.lb
        lo, hi, leaf_hi, x = self.lo[keep], self.hi[keep], leaf_hi[keep], self.x[keep]
        self.ub = min(self.ub, float(leaf_hi.max()))
        # split the leaves with the largest upper bound
        room = max(0, self.max_leaves - lo.shape[0])
        n_split = min(room, lo.shape[0], self.split_per_round)
        if n_split > 0:
            order = torch.argsort(leaf_hi, descending=True)
            sel = order[:n_split]
            rest = order[n_split:]
            glo, ghi = self._grad(lo[sel], hi[sel])
            width = hi[sel] - lo[sel]
            score = (glo.abs() + ghi.abs()) * width
            score = torch.where(width > 0, score, torch.full_like(score, -1.0))
            dim = torch.argmax(score, dim=1)
            rows = torch.arange(n_split, device=self.device)
            m = 0.5 * (lo[sel][rows, dim] + hi[sel][rows, dim])
            a_lo, a_hi = lo[sel].clone(), hi[sel].clone()
            b_lo, b_hi = lo[sel].clone(), hi[sel].clone()
            a_hi[rows, dim] = m
            b_lo[rows, dim] = m
            self.lo = torch.cat([lo[rest], a_lo, b_lo])
            self.hi = torch.cat([hi[rest], a_hi, b_hi])
            xs = x[sel]
            self.x = torch.cat([x[rest], torch.minimum(torch.maximum(xs, a_lo), a_hi),
                                torch.minimum(torch.maximum(xs, b_lo), b_hi)])
        else:
            self.lo, self.hi, self.x = lo, hi, x
        torch.cuda.synchronize(self.device)
        self._elapsed += time.perf_counter() - t0
        self.round += 1
        gap = (self.ub - self.lb) / max(abs(self.lb), 1e-300)
        rec = RoundRecord(self.round, self._elapsed, self.ub, self.lb, gap, int(self.lo.shape[0]))
        self.history.append(rec)
        return rec

    def run(self, rounds: int) -> List[RoundRecord]:
        for _ in range(rounds):
            self.step()
        return self.history

    # -------------------------------------------------------------- checkpoint
    def save(self, path: str):
        np.savez(path, lo=self.lo.cpu().numpy(), hi=self.hi.cpu().numpy(), x=self.x.cpu().numpy(),
                 ub=self.ub, lb=self.lb, round=self.round, elapsed=self._elapsed,
                 step_frac=self.step_frac)

    @classmethod
    def load(cls, case: Case, path: str, **kw) -> "Bisection":
        z = np.load(path)
        b = cls(case, z["lo"], z["hi"], **kw)
        b.ub, b.lb = float(z["ub"]), float(z["lb"])
        b.round = int(z["round"])
        b._elapsed = float(z["elapsed"])
        b.x = torch.as_tensor(z["x"], dtype=torch.float64, device=b.device)
        b.step_frac = float(z["step_frac"])
        return b


__all__ = ["Bisection", "RoundRecord"]
