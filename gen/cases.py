"""Seeded synthetic cases with the shapes of the GO3 instances (paper Table I).

The GO3 competition instances used in the paper are not available here, so every
workload is drawn from a seeded generator with the sizes of the paper's cases:

* network: a random recursive spanning tree over a seeded permutation of the
  buses plus uniform random extra edges (no self loops, no parallel lines),
  reactances lognormal(mu=-2.3, sigma=0.5) p.u.  The 5-bus case is the fixed
  ring 0-1-2-3-4-0 plus the chord 1-3 with reactances U[0.05, 0.5];
* devices: generators and flexible loads on distinct random buses, generator
  box [0, Pmax] with Pmax ~ U[50, 500] MW and cost ~ U[10, 60] $/MWh, load box
  [0.7, 1.0] x nominal with nominal ~ U[30, 200] MW and value ~ U[40, 120] $/MWh;
* ratings: max(1.2 |f_l|, 1 MW) where f_l is the DC base flow at the box
  midpoint (single slack bus 0 absorbing the mismatch); a few lines are
  tightened to 0.8 |f_l|;
* contingencies: the non-islanding (non-bridge) N-1 line outages, optionally a
  seeded subset of them.

The DC angle solve used for the ratings is part of *drawing* the input data; the
bound computations on both sides (oracle and CUDA library) build their own
sensitivities and share nothing with this module.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

ZETA_INJ = 1.0e4  # $/MW, nodal imbalance penalty
ZETA_F = 1.0e3    # $/MW, base and contingency overflow penalty

# (n_bus, n_line, n_gen, n_load, n_ctg or None for "all non-bridges")
CONFIG_SIZES = {
    0: (5, 6, 2, 3, None),
    1: (118, 186, 54, 99, None),
    2: (2000, 3200, 500, 1200, 2500),
    3: (8316, 10500, 1100, 5000, 5000),
    # profiling size: PTDF rows larger than the 129 MB L2, a few ms per bound
    5: (5000, 7000, 660, 3000, 4000),
}
RAGGED_SIZES = (73, 300, 500, 1000, 2000)


@dataclasses.dataclass
class Case:
    """One network with its devices, prices, contingency list and boxes.

    Devices are ordered generators first, then loads, in every box array.
    Piecewise-linear curves are stored as flattened per-device segments:
    device i owns segments ``seg_ptr[i]:seg_ptr[i+1]`` with slope ``a`` (>= 0)
    and segment start ``b`` (increasing).
    """

    name: str
    n_bus: int
    slack: int
    line_from: np.ndarray  # int32 [n_line]
    line_to: np.ndarray    # int32 [n_line]
    reactance: np.ndarray  # float64 [n_line], p.u. > 0
    rating: np.ndarray     # float64 [n_line], MW >= 0
    gen_bus: np.ndarray    # int32 [n_gen]
    gen_nseg: np.ndarray   # int32 [n_gen]
    gen_slope: np.ndarray  # float64 [sum gen_nseg], $/MWh
    gen_bkpt: np.ndarray   # float64 [sum gen_nseg], MW
    load_bus: np.ndarray   # int32 [n_load]
    load_nseg: np.ndarray
    load_slope: np.ndarray
    load_bkpt: np.ndarray
    zeta_inj: float
    zeta_f: float
    ctg_line: np.ndarray   # int32 [n_ctg]
    box_lo: np.ndarray     # float64 [n_box, n_gen + n_load]
    box_hi: np.ndarray
    rating_ctg: Optional[np.ndarray] = None

    @property
    def n_line(self) -> int:
        return int(self.line_from.shape[0])

    @property
    def n_gen(self) -> int:
        return int(self.gen_bus.shape[0])

    @property
    def n_load(self) -> int:
        return int(self.load_bus.shape[0])

    @property
    def n_dev(self) -> int:
        return self.n_gen + self.n_load

    @property
    def n_ctg(self) -> int:
        return int(self.ctg_line.shape[0])

    @property
    def n_box(self) -> int:
        return int(self.box_lo.shape[0])

    def active_buses(self) -> np.ndarray:
        """Buses that carry at least one device, slack excluded (sorted)."""
        s = set(self.gen_bus.tolist()) | set(self.load_bus.tolist())
        s.discard(self.slack)
        return np.array(sorted(s), dtype=np.int32)

    def with_boxes(self, lo: np.ndarray, hi: np.ndarray) -> "Case":
        return dataclasses.replace(self, box_lo=np.ascontiguousarray(lo, np.float64),
                                   box_hi=np.ascontiguousarray(hi, np.float64))


# ----------------------------------------------------------------------------
# graph helpers (no interval arithmetic here)
# ----------------------------------------------------------------------------

def find_bridges(n_bus: int, line_from: Sequence[int], line_to: Sequence[int]) -> np.ndarray:
    """Boolean mask of bridge lines (removal disconnects the graph).

    Iterative Tarjan low-link DFS; parallel lines are handled by skipping only
    the tree edge's own index, not every edge to the parent.
    """
    n_line = len(line_from)
    adj: List[List[tuple]] = [[] for _ in range(n_bus)]
    for e in range(n_line):
        a, b = int(line_from[e]), int(line_to[e])
        adj[a].append((b, e))
        adj[b].append((a, e))
    disc = [-1] * n_bus
    low = [0] * n_bus
    is_bridge = np.zeros(n_line, dtype=bool)
    t = 0
    for root in range(n_bus):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = t
        t += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            v, pe, it = stack[-1]
            advanced = False
            for (w, e) in it:
                if e == pe:
                    continue
                if disc[w] < 0:
                    disc[w] = low[w] = t
                    t += 1
                    stack.append((w, e, iter(adj[w])))
                    advanced = True
                    break
                low[v] = min(low[v], disc[w])
            if advanced:
                continue
            stack.pop()
            if stack:
                u = stack[-1][0]
                low[u] = min(low[u], low[v])
                if low[v] > disc[u]:
                    is_bridge[pe] = True
    return is_bridge


def _random_network(n_bus: int, n_line: int, rng: np.random.Generator):
    if n_line < n_bus - 1:
        raise ValueError("need at least a spanning tree")
    perm = rng.permutation(n_bus)
    seen = set()
    fr, to = [], []
    for i in range(1, n_bus):
        j = int(rng.integers(0, i))
        a, b = int(perm[i]), int(perm[j])
        seen.add((min(a, b), max(a, b)))
        fr.append(a)
        to.append(b)
    max_edges = n_bus * (n_bus - 1) // 2
    if n_line > max_edges:
        raise ValueError("too many lines for a simple graph")
    while len(fr) < n_line:
        a, b = (int(v) for v in rng.integers(0, n_bus, size=2))
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in seen:
            continue
        seen.add(key)
        fr.append(a)
        to.append(b)
    x = rng.lognormal(mean=-2.3, sigma=0.5, size=n_line)
    return np.array(fr, np.int32), np.array(to, np.int32), x


def _dc_midpoint_flows(n_bus, slack, fr, to, x, inj):
    """DC base flows for a nodal injection vector (slack absorbs the mismatch).

    Only used to draw line ratings.  Sparse reduced-Laplacian angle solve.
    """
    b = 1.0 / x
    keep = np.array([i for i in range(n_bus) if i != slack])
    pos = -np.ones(n_bus, dtype=np.int64)
    pos[keep] = np.arange(keep.size)
    try:
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        rows, cols, vals = [], [], []
        for e in range(fr.size):
            i, j = int(fr[e]), int(to[e])
            for (p, q, v) in ((i, i, b[e]), (j, j, b[e]), (i, j, -b[e]), (j, i, -b[e])):
                if pos[p] >= 0 and pos[q] >= 0:
                    rows.append(pos[p]); cols.append(pos[q]); vals.append(v)
        Y = sp.csc_matrix((vals, (rows, cols)), shape=(keep.size, keep.size))
        th_r = spla.spsolve(Y, inj[keep])
    except ImportError:  # dense fallback for tiny cases
        Y = np.zeros((keep.size, keep.size))
        for e in range(fr.size):
            i, j = pos[int(fr[e])], pos[int(to[e])]
            if i >= 0:
                Y[i, i] += b[e]
            if j >= 0:
                Y[j, j] += b[e]
            if i >= 0 and j >= 0:
                Y[i, j] -= b[e]
                Y[j, i] -= b[e]
        th_r = np.linalg.solve(Y, inj[keep])
    th = np.zeros(n_bus)
    th[keep] = th_r
    return b * (th[fr] - th[to])


def _pwl(rng, n_dev, pmax, lo_slope, hi_slope, nseg, convex):
    """Per-device PWL curves: n_seg equal-width segments starting at 0."""
    nsegs = np.full(n_dev, nseg, dtype=np.int32)
    slopes = np.empty(n_dev * nseg)
    bk = np.empty(n_dev * nseg)
    for i in range(n_dev):
        s = np.sort(rng.uniform(lo_slope, hi_slope, size=nseg))
        if not convex:
            s = s[::-1]
        slopes[i * nseg:(i + 1) * nseg] = s
        bk[i * nseg:(i + 1) * nseg] = pmax[i] * np.arange(nseg) / nseg
    return nsegs, slopes, bk


def make_network_case(name: str, n_bus: int, n_line: int, n_gen: int, n_load: int,
                      seed: int, n_ctg: Optional[int] = None, n_seg: int = 1,
                      n_tighten: Optional[int] = None, ring5: bool = False,
                      topology=None, slack: int = 0) -> Case:
    """Draw one network case with a single root box.  ``topology`` = (from,
    to) fixes the lines (reactances are still drawn)."""
    rng = np.random.default_rng(seed)
    if topology is not None:
        fr = np.asarray(topology[0], np.int32)
        to = np.asarray(topology[1], np.int32)
        x = np.exp(rng.normal(-2.3, 0.5, size=fr.size))
    elif ring5:
        fr = np.array([0, 1, 2, 3, 4, 1], np.int32)
        to = np.array([1, 2, 3, 4, 0, 3], np.int32)
        x = rng.uniform(0.05, 0.5, size=6)
    else:
        fr, to, x = _random_network(n_bus, n_line, rng)
    gen_bus = np.sort(rng.choice(n_bus, size=n_gen, replace=False)).astype(np.int32)
    load_bus = np.sort(rng.choice(n_bus, size=n_load, replace=False)).astype(np.int32)
    pmax = rng.uniform(50.0, 500.0, size=n_gen)
    nominal = rng.uniform(30.0, 200.0, size=n_load)
    gen_nseg, gen_slope, gen_bkpt = _pwl(rng, n_gen, pmax, 10.0, 60.0, n_seg, convex=True)
    load_nseg, load_slope, load_bkpt = _pwl(rng, n_load, nominal, 40.0, 120.0, n_seg, convex=False)

    lo = np.concatenate([np.zeros(n_gen), 0.7 * nominal])
    hi = np.concatenate([pmax, 1.0 * nominal])

    mid = 0.5 * (lo + hi)
    inj = np.zeros(n_bus)
    np.add.at(inj, gen_bus, mid[:n_gen])
    np.add.at(inj, load_bus, -mid[n_gen:])
    f = _dc_midpoint_flows(n_bus, slack, fr, to, x, inj)
    absf = np.abs(f)
    factor = np.full(fr.size, 1.2)
    if ring5:
        tight = np.argsort(-absf, kind="stable")[:2]
    else:
        k = n_tighten if n_tighten is not None else max(2, math.ceil(0.01 * fr.size))
        tight = rng.choice(fr.size, size=k, replace=False)
    factor[tight] = 0.8
    rating = np.maximum(factor * absf, 1.0)

    bridges = find_bridges(n_bus, fr, to)
    ctg = np.flatnonzero(~bridges).astype(np.int32)
    if n_ctg is not None and n_ctg < ctg.size:
        ctg = np.sort(rng.permutation(ctg)[:n_ctg]).astype(np.int32)
    return Case(name=name, n_bus=n_bus, slack=slack, line_from=fr, line_to=to,
                reactance=x, rating=rating, gen_bus=gen_bus, gen_nseg=gen_nseg,
                gen_slope=gen_slope, gen_bkpt=gen_bkpt, load_bus=load_bus,
                load_nseg=load_nseg, load_slope=load_slope, load_bkpt=load_bkpt,
                zeta_inj=ZETA_INJ, zeta_f=ZETA_F, ctg_line=ctg,
                box_lo=lo[None, :].copy(), box_hi=hi[None, :].copy())


def make_two_core_case(seed: int = 1200) -> Case:
    """Two meshed cores joined by a path of bridges, radial feeders hanging off
    both, and the slack at the end of a feeder: a small network whose
    2-edge-connected structure has several parts with inner lines."""
    core_a = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (1, 4), (2, 5)]
    core_b = [(10, 11), (11, 12), (12, 13), (13, 14), (14, 10), (11, 13)]
    core_c = [(20, 21), (21, 22), (22, 20)]
    path = [(3, 6), (6, 7), (7, 10), (12, 18), (18, 20)]
    feeders = [(0, 8), (8, 9), (9, 24), (5, 15), (15, 16), (16, 17), (14, 19), (19, 23),
               (21, 25), (25, 26), (6, 27)]
    lines = core_a + core_b + core_c + path + feeders
    fr = np.array([a for a, _ in lines], np.int32)
    to = np.array([b for _, b in lines], np.int32)
    return make_network_case("two-core", 28, len(lines), 8, 14, seed=seed, topology=(fr, to),
                             slack=24)


def time_index_boxes(case: Case, n_box: int, seed: int) -> Case:
    """Boxes standing in for time indices: loads scaled by a seeded U[0.8, 1.2]."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.8, 1.2, size=n_box)
    lo = np.repeat(case.box_lo, n_box, axis=0)
    hi = np.repeat(case.box_hi, n_box, axis=0)
    ng = case.n_gen
    lo[:, ng:] *= s[:, None]
    hi[:, ng:] *= s[:, None]
    return case.with_boxes(lo, hi)


def split_boxes(lo: np.ndarray, hi: np.ndarray, levels: int, rng: np.random.Generator):
    """Tile a box into 2**levels sub-boxes by halving one seeded dimension per level."""
    los, his = [np.asarray(lo, np.float64)], [np.asarray(hi, np.float64)]
    for _ in range(levels):
        nl, nh = [], []
        for a, b in zip(los, his):
            widths = b - a
            cand = np.flatnonzero(widths > 0)
            d = int(rng.choice(cand))
            m = 0.5 * (a[d] + b[d])
            a1, b1 = a.copy(), b.copy()
            b1[d] = m
            a2, b2 = a.copy(), b.copy()
            a2[d] = m
            nl += [a1, a2]
            nh += [b1, b2]
        los, his = nl, nh
    return np.stack(los), np.stack(his)


def make_config(cfg: int, n_box: int = 1, n_seg: int = 1) -> Case:
    """The seeded case of synthetic workload ``cfg`` (0..3, 5); seed 1000 + cfg."""
    n_bus, n_line, n_gen, n_load, n_ctg = CONFIG_SIZES[cfg]
    names = {0: "ring5", 1: "mesh118", 2: "mesh2000", 3: "mesh8316", 5: "mesh5000"}
    c = make_network_case(names[cfg], n_bus, n_line, n_gen, n_load, seed=1000 + cfg,
                          n_ctg=n_ctg, n_seg=n_seg, ring5=(cfg == 0))
    if n_box > 1:
        c = time_index_boxes(c, n_box, seed=2000 + cfg)
    return c


def make_case(cfg: int, **kw) -> Case:
    return make_config(cfg, **kw)


def make_ragged_batch(n_net: int = 64, n_sub: int = 16, seed: int = 1004,
                      sizes: Sequence[int] = RAGGED_SIZES) -> List[Case]:
    """Networks of uneven size, each with all its non-bridge contingencies and
    ``n_sub`` sub-boxes from seeded bisection of its root box."""
    rng = np.random.default_rng(seed)
    out = []
    levels = int(round(math.log2(n_sub)))
    if 2 ** levels != n_sub:
        raise ValueError("n_sub must be a power of two")
    for i in range(n_net):
        nb = int(rng.choice(sizes))
        nl = int(round(1.6 * nb))
        ng = max(1, int(round(0.25 * nb)))
        nd = max(1, int(round(0.6 * nb)))
        c = make_network_case(f"ragged{i}_{nb}", nb, nl, ng, nd, seed=int(rng.integers(1 << 30)))
        lo, hi = split_boxes(c.box_lo[0], c.box_hi[0], levels, rng)
        out.append(c.with_boxes(lo, hi))
    return out
