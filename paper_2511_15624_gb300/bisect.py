"""Gradient-guided input-box bisection on top of the certified bound.

The paper bounds max f over the whole input box with one IBP pass and names
branch-and-bound over the input domain as future work (Sec. I, Sec. V).  This
driver keeps a frontier of leaf boxes that tile the part of the root box that
may still hold the maximiser:

* UB = max over leaves of obj_hi is a certified upper bound of max f over the
  root box (leaves dropped below hold max f <= their obj_hi < LB <= max f);
* LB = max over evaluated points y of obj_lo of the zero-width box at y, a
  certified lower bound of f(y) <= max f.  Each leaf carries an accepted
  point x (its centre at first), the certified value at x and a step s in
  (0, 1].  Every round evaluates the proposal y made in the round before; y
  replaces x when its value is higher (s grows by 1.5, else s halves).  The
  next proposal is a conditional-gradient step inside the leaf: with g the
  gradient of f at x (the adjoint of the zero-width box), the leaf vertex v
  that maximises g.v, and y = x + s (v - x).  f is concave, so the accepted
  points climb;
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
        n = self.lo.shape[0]
        self.x = 0.5 * (self.lo + self.hi)  # accepted point per leaf
        self.fx = torch.full((n,), -float("inf"), dtype=torch.float64, device=self.device)
        self.y = self.x.clone()             # proposal, evaluated in the next round
        self.s = torch.full((n,), 0.5, dtype=torch.float64, device=self.device)
        self.ub = float("inf")
        self.lb = -float("inf")
        self.round = 0
        self.history: List[RoundRecord] = []
        self._t0 = None
        self._elapsed = 0.0

    def _sync(self):
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

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
        self._sync()
        t0 = time.perf_counter()
        n = self.lo.shape[0]
        both_lo = torch.cat([self.lo, self.y])
        both_hi = torch.cat([self.hi, self.y])
        obj_lo, obj_hi = self._bound(both_lo, both_hi)
        leaf_hi = obj_hi[:n]
        fy = obj_lo[n:]
        self.lb = max(self.lb, float(fy.max()))
        # accept the proposals that improved their leaf's point
        better = fy > self.fx
        self.x = torch.where(better[:, None], self.y, self.x)
        self.fx = torch.where(better, fy, self.fx)
        self.s = torch.where(better, torch.clamp(1.5 * self.s, max=1.0), 0.5 * self.s)
        # next proposals: conditional-gradient step towards the best vertex
        gxl, gxh = self._grad(self.x, self.x)
        g = gxl + gxh
        v = torch.where(g > 0, self.hi, torch.where(g < 0, self.lo, self.x))
        self.y = self.x + self.s[:, None] * (v - self.x)
        keep = leaf_hi >= self.lb
        lo, hi, leaf_hi = self.lo[keep], self.hi[keep], leaf_hi[keep]
        x, fx, y, sv = self.x[keep], self.fx[keep], self.y[keep], self.s[keep]
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

            def clamp(v, l, h):
                return torch.minimum(torch.maximum(v, l), h)

            xs, ys, fs, ss = x[sel], y[sel], fx[sel], sv[sel]
            xa, xb = clamp(xs, a_lo, a_hi), clamp(xs, b_lo, b_hi)
            # the child that does not hold x gets the projection, not yet evaluated
            ninf = torch.full_like(fs, -float("inf"))
            fa = torch.where((xa == xs).all(dim=1), fs, ninf)
            fb = torch.where((xb == xs).all(dim=1), fs, ninf)
            self.x = torch.cat([x[rest], xa, xb])
            self.fx = torch.cat([fx[rest], fa, fb])
            self.y = torch.cat([y[rest], clamp(ys, a_lo, a_hi), clamp(ys, b_lo, b_hi)])
            self.s = torch.cat([sv[rest], ss, ss])
        else:
            self.lo, self.hi, self.x, self.fx, self.y, self.s = lo, hi, x, fx, y, sv
        self._sync()
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
                 fx=self.fx.cpu().numpy(), y=self.y.cpu().numpy(), s=self.s.cpu().numpy(),
                 ub=self.ub, lb=self.lb, round=self.round, elapsed=self._elapsed)

    @classmethod
    def load(cls, case: Case, path: str, **kw) -> "Bisection":
        z = np.load(path)
        b = cls(case, z["lo"], z["hi"], **kw)
        b.ub, b.lb = float(z["ub"]), float(z["lb"])
        b.round = int(z["round"])
        b._elapsed = float(z["elapsed"])
        for name in ("x", "fx", "y", "s"):
            setattr(b, name, torch.as_tensor(z[name], dtype=torch.float64, device=b.device))
        return b


__all__ = ["Bisection", "RoundRecord"]
