"""Gradient-guided input-box bisection on top of the certified bounds.

The paper bounds max f over the whole input box with one IBP pass and names
branch-and-bound over the input domain as future work (Sec. I, Sec. V).  This
driver keeps a frontier of leaf boxes that tile the part of the root box that
may still hold the maximiser:

* UB = max over leaves of the leaf's certified upper bound of max f: obj_hi of
  ibp_bound (bound="ibp"), or the smaller of that and the linear relaxation
  bound of ibp_bound_linear (bound="linear"; each child continues the
  parent's slopes, so a round refines rather than restarts).  Leaves whose
  bound falls below LB are dropped: they cannot hold the maximiser;
* LB = max over evaluated points y of a certified lower bound of f(y): at a
  zero-width box the IBP bound is f(y) itself, so obj_hi(y) - err_hi(y) <=
  f(y) (obj_err bounds the distance of obj_hi from the exact IBP value, which
  the FP64 refinement makes FP64-small); with every radius 0 the paper's
  two-part contingency interval is exact, so points go through
  ibp_bound_paper.  Each leaf carries an accepted point
  x (its centre at first), the certified value at x and a step s in (0, 1].
  Every round evaluates the proposal y made in the round before; y replaces x
  when its value is higher (s grows by 1.5, else s halves).  The next
  proposal is a conditional-gradient step inside the leaf: with g the
  gradient of f at x (the adjoint of the zero-width box), the leaf vertex v
  that maximises g.v, and y = x + s (v - x); with bound="linear" the
  relaxation's averaged primal point of the leaf is evaluated too;
* each round splits up to ``split_per_round`` leaves with the largest upper
  bound (default: every leaf, until the frontier holds ``max_leaves``) at the
  midpoint of the coordinate with the largest
  (|d obj_hi / d lo_i| + |d obj_hi / d hi_i|) * width_i.

f is concave on the box (concave value curves, convex cost curves, convex
penalties), so max f over a box is a linear program, whose dual
ibp_bound_linear optimises: the leaf that holds the maximiser keeps the root's
LP value whatever the splits, and with linear leaves UB falls only as the
relaxation converges (bisection then prunes leaves below LB, but does not
lower the top leaf).  IBP leaves lower UB slowly: IBP's excess comes from the
same devices entering many penalty terms, which splitting one coordinate at a
time barely removes.

``batched=True`` bounds all leaves (and points) of a round in one call of
each kind; ``batched=False`` makes one call per box with the same rules.  The
two use different kernels (one box or many), whose results differ in the last
bits of obj_lo and, for obj_hi, within FP64 rounding; a tie between two leaves'
bounds or two points' values can then break differently and the frontiers
part.  The frontier (boxes, UB, LB, round) can be saved and reloaded.
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
    seconds: float       # wall time of all rounds so far
    ub: float
    lb: float
    gap: float           # (ub - lb) / |lb|
    n_leaves: int
    bound_seconds: float = 0.0  # this round's time inside the library calls
    round_seconds: float = 0.0  # this round's wall time


class Bisection:
    def __init__(self, case: Case, root_lo, root_hi, max_leaves: int = 256,
                 batched: bool = True, device: Optional[torch.device] = None,
                 split_per_round: Optional[int] = None, bound: str = "ibp",
                 linear_iters: int = 1000, linear_root_iters: Optional[int] = None,
                 primal_weight: float = 0.01):
        self.case = case
        self.device = device or torch.device("cuda", case.device)
        lo = torch.as_tensor(np.atleast_2d(root_lo), dtype=torch.float64, device=self.device)
        hi = torch.as_tensor(np.atleast_2d(root_hi), dtype=torch.float64, device=self.device)
        self.lo, self.hi = lo.clone(), hi.clone()
        self.max_leaves = int(max_leaves)
        self.split_per_round = int(split_per_round) if split_per_round else self.max_leaves
        self.batched = bool(batched)
        if bound not in ("ibp", "linear"):
            raise ValueError("bound must be 'ibp' or 'linear'")
        self.bound_kind = bound
        self.linear_iters = int(linear_iters)
        self.linear_root_iters = int(linear_root_iters or 10 * linear_iters)
        self.primal_weight = float(primal_weight)
        n = self.lo.shape[0]
        self.x = 0.5 * (self.lo + self.hi)  # accepted point per leaf
        self.fx = torch.full((n,), -float("inf"), dtype=torch.float64, device=self.device)
        self.y = self.x.clone()             # proposal, evaluated in the next round
        self.s = torch.full((n,), 0.5, dtype=torch.float64, device=self.device)
        self.ub = float("inf")
        self.lb = -float("inf")
        self.round = 0
        self.history: List[RoundRecord] = []
        self._elapsed = 0.0
        self._tb = 0.0
        self._lin_ready = False  # the case holds linear state for the current leaves
        self._xlin = None        # the relaxation's primal points of the current leaves

    def _sync(self):
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

    def _timed(self, fn, *args, **kw):
        self._sync()
        t0 = time.perf_counter()
        out = fn(*args, **kw)
        self._sync()
        self._tb += time.perf_counter() - t0
        return out

    # -------------------------------------------------------------- bounds
    def _bound(self, lo, hi):
        """obj_hi of every leaf box."""
        if self.batched:
            return self._timed(self.case.bound, lo, hi)[1]
        return torch.cat([self._timed(self.case.bound, lo[j:j + 1], hi[j:j + 1])[1]
                          for j in range(lo.shape[0])])

    def _points(self, y):
        """Certified lower bounds obj_hi - err_hi of f at the points y.  At a
        zero-width box every radius is 0, so the paper's two-part contingency
        interval (ibp_bound_paper, O(n_ctg n_line)) is exact there and the
        contingency kernel is not needed."""
        fn = getattr(self.case, "bound_paper", None) or self.case.bound
        if self.batched:
            _, hi, err = self._timed(fn, y, y)
            return hi - err[:, 0]
        out = []
        for j in range(y.shape[0]):
            _, hi, err = self._timed(fn, y[j:j + 1], y[j:j + 1])
            out.append(hi - err[:, 0])
        return torch.cat(out)

    def _grad(self, lo, hi):
        ones = torch.ones(lo.shape[0], dtype=torch.float64, device=self.device)
        if self.batched:
            return self._timed(self.case.backward, lo, hi, ones)
        gl, gh = [], []
        for j in range(lo.shape[0]):
            a, b = self._timed(self.case.backward, lo[j:j + 1], hi[j:j + 1], ones[j:j + 1])
            gl.append(a)
            gh.append(b)
        return torch.cat(gl), torch.cat(gh)

    def _linear(self, lo, hi):
        """Linear relaxation bounds of the leaves (continuing their slopes) and
        the relaxation's primal points."""
        warm = self._lin_ready
        iters = self.linear_iters if warm else self.linear_root_iters
        if not warm and not self.batched and lo.shape[0] > 1:
            # a reloaded frontier: hold zero slopes for every leaf, then continue each
            self._timed(self.case.bound_linear, lo, hi, 0, self.primal_weight)
            warm = True
        if self.batched or lo.shape[0] == 1:
            ub, _, xp = self._timed(self.case.bound_linear, lo, hi, iters, self.primal_weight, None, warm)
        else:
            # one box per call, each continuing its own held state
            ubs, xps = [], []
            for j in range(lo.shape[0]):
                if warm:
                    u, _, x = self._timed(self.case.bound_linear, lo[j:j + 1], hi[j:j + 1], iters,
                                          self.primal_weight, None, True, j)
                else:  # a fresh root: one box
                    u, _, x = self._timed(self.case.bound_linear, lo[j:j + 1], hi[j:j + 1], iters,
                                          self.primal_weight)
                ubs.append(u)
                xps.append(x)
            ub, xp = torch.cat(ubs), torch.cat(xps)
        self._lin_ready = True
        return ub, xp

    # -------------------------------------------------------------- rounds
    def step(self) -> RoundRecord:
        self._sync()
        t0 = time.perf_counter()
        self._tb = 0.0
        n = self.lo.shape[0]
        pts = [self.y]
        leaf_hi = self._bound(self.lo, self.hi)
        if self.bound_kind == "linear":
            lub, xp = self._linear(self.lo, self.hi)
            leaf_hi = torch.minimum(leaf_hi, lub)
            self._xlin = xp
            pts.append(xp)
        pv = self._points(torch.cat(pts))
        fy = pv[:n]
        self.lb = max(self.lb, float(pv.max()))
        # accept the proposals that improved their leaf's point
        better = fy > self.fx
        self.x = torch.where(better[:, None], self.y, self.x)
        self.fx = torch.where(better, fy, self.fx)
        if self.bound_kind == "linear":
            fl = pv[n:]
            bl = fl > self.fx
            self.x = torch.where(bl[:, None], self._xlin, self.x)
            self.fx = torch.where(bl, fl, self.fx)
            better = better | bl
        self.s = torch.where(better, torch.clamp(1.5 * self.s, max=1.0), 0.5 * self.s)
        # next proposals: conditional-gradient step towards the best vertex
        gxl, gxh = self._grad(self.x, self.x)
        g = gxl + gxh
        v = torch.where(g > 0, self.hi, torch.where(g < 0, self.lo, self.x))
        self.y = self.x + self.s[:, None] * (v - self.x)
        keep = leaf_hi >= self.lb
        if not bool(keep.any()):
            # cannot happen in exact arithmetic (the leaf holding the best point
            # bounds it from above); keep the top leaf rather than an empty frontier
            keep = leaf_hi == leaf_hi.max()
        kidx = torch.nonzero(keep).flatten()
        lo, hi, leaf_hi = self.lo[keep], self.hi[keep], leaf_hi[keep]
        x, fx, y, sv = self.x[keep], self.fx[keep], self.y[keep], self.s[keep]
        self.ub = min(self.ub, float(leaf_hi.max()))
        # split the leaves with the largest upper bound
        room = max(0, self.max_leaves - lo.shape[0])
        n_split = min(room, lo.shape[0], self.split_per_round)
        parent = kidx
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
            parent = torch.cat([kidx[rest], kidx[sel], kidx[sel]])

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
        if self.bound_kind == "linear":
            # children continue their parent's slopes
            self._timed(self.case.linear_inherit, parent.cpu().numpy().astype(np.int32))
        self._sync()
        dt = time.perf_counter() - t0
        self._elapsed += dt
        self.round += 1
        gap = (self.ub - self.lb) / max(abs(self.lb), 1e-300)
        rec = RoundRecord(self.round, self._elapsed, self.ub, self.lb, gap, int(self.lo.shape[0]),
                          self._tb, dt)
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
