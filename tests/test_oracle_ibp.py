"""Pins for the oracle's IBP bound (Sec. III, appendix eq. (ibp_f)):
exact ranges by vertex enumeration, soundness at vertices and random points,
an LP optimum, point evaluation by brute-force re-solves, the penalty-map case
table, the imbalance closed form, the ReLU-chain costs and finite differences
of the hand adjoint."""
import itertools

import numpy as np
import pytest

import oracle as O
from gen import make_config, split_boxes
from tests._brute import objective_brute, pwl_direct


def _vertices(lo, hi):
    n = lo.size
    for bits in itertools.product((0, 1), repeat=n):
        m = np.array(bits, bool)
        yield np.where(m, hi, lo)


def test_flow_intervals_are_exact_ranges(cases):
    """Each contingency/base flow is affine in the device powers and every device
    sits on one bus, so IBP's [c - r, c + r] is the exact range: the vertex
    extremes must hit it."""
    c = cases(0)
    s = O.sensitivities(c)
    cb, rb = O.bus_box(c, c.box_lo, c.box_hi)
    cent, rad = O.all_ctg_flows(c, s, cb, rb)
    vmin = np.full((c.n_ctg, c.n_line), np.inf)
    vmax = -vmin
    for x in _vertices(c.box_lo[0], c.box_hi[0]):
        p, _ = O.bus_box(c, x[None], x[None])
        f = s.phi @ p[0]
        for k in range(c.n_ctg):
            fk = f + s.lodf[:, k] * f[c.ctg_line[k]]
            vmin[k] = np.minimum(vmin[k], fk)
            vmax[k] = np.maximum(vmax[k], fk)
    scale = np.abs(cent[0]) + rad[0] + 1.0
    np.testing.assert_allclose(cent[0] - rad[0], vmin, rtol=0, atol=1e-12 * scale.max())
    np.testing.assert_allclose(cent[0] + rad[0], vmax, rtol=0, atol=1e-12 * scale.max())
    # the outaged line's flow is exactly zero
    assert np.all(cent[0][np.arange(c.n_ctg), c.ctg_line] == 0.0)
    assert np.all(rad[0][np.arange(c.n_ctg), c.ctg_line] == 0.0)


def test_random_vertices_inside_and_extreme_attained(cases):
    c = cases(1)
    s = O.sensitivities(c)
    cb, rb = O.bus_box(c, c.box_lo, c.box_hi)
    rng = np.random.default_rng(1)
    pk = rng.integers(0, c.n_ctg, 40)
    pl = rng.integers(0, c.n_line, 40)
    cent, rad = O.ctg_flows(c, s, cb, rb, pk, pl)
    ng = c.n_gen
    lo, hi = c.box_lo[0], c.box_hi[0]
    for i in range(pk.size):
        k, l = pk[i], pl[i]
        h = s.phi[l] + s.lodf[l, k] * s.phi[c.ctg_line[k]]
        w = np.concatenate([h[c.gen_bus], -h[c.load_bus]])  # flow per device MW
        xmax = np.where(w >= 0, hi, lo)
        xmin = np.where(w >= 0, lo, hi)
        assert abs(w @ xmax - (cent[0, i] + rad[0, i])) <= 1e-10 * (abs(cent[0, i]) + rad[0, i] + 1)
        assert abs(w @ xmin - (cent[0, i] - rad[0, i])) <= 1e-10 * (abs(cent[0, i]) + rad[0, i] + 1)
        for _ in range(20):
            x = np.where(rng.random(lo.size) < 0.5, lo, hi)
            v = w @ x
            assert cent[0, i] - rad[0, i] - 1e-9 <= v <= cent[0, i] + rad[0, i] + 1e-9
    del ng


def test_objective_sound_at_all_vertices_and_exact_min(cases):
    """f is concave (concave PWL values, convex PWL costs, -|affine| penalties),
    so its minimum over the box sits at a vertex: lo <= min_vertices f, and
    every vertex value lies inside [lo, hi]."""
    c = cases(0)
    s = O.sensitivities(c)
    b = O.bound(c, s)
    vals = [O.objective_point(c, s, x) for x in _vertices(c.box_lo[0], c.box_hi[0])]
    assert b.lo[0] <= min(vals) + 1e-9 * abs(min(vals))
    assert b.hi[0] >= max(vals) - 1e-9 * abs(max(vals))


@pytest.mark.parametrize("cfg,npts", [(0, 100_000), (1, 100_000)])
def test_objective_sound_random_points(cases, cfg, npts):
    c = cases(cfg)
    s = O.sensitivities(c)
    b = O.bound(c, s)
    rng = np.random.default_rng(100 + cfg)
    lo, hi = c.box_lo[0], c.box_hi[0]
    ng = c.n_gen
    # vectorised f over many points (linear costs in these configs)
    assert np.all(c.gen_nseg == 1) and np.all(c.load_nseg == 1)
    W = O.imbalance_matrix(c, s.phi)
    rating = c.rating
    fmin, fmax = np.inf, -np.inf
    batch = 2000 if cfg == 0 else 500
    done = 0
    while done < npts:
        n = min(batch, npts - done)
        X = lo + rng.random((n, lo.size)) * (hi - lo)
        P, _ = O.bus_box(c, X, X)
        F = P @ s.phi.T
        s_inj = np.abs(P @ W.T).sum(axis=1)
        s_fb = np.maximum(np.abs(F) - rating, 0).sum(axis=1)
        Pc = F[:, None, :] + s.lodf.T[None] * F[:, c.ctg_line][:, :, None]
        s_fc = np.maximum(np.abs(Pc) - rating, 0).sum(axis=(1, 2))
        val = X[:, ng:] @ c.load_slope - X[:, :ng] @ c.gen_slope
        f = val - c.zeta_inj * s_inj - c.zeta_f * (s_fb + s_fc)
        fmin = min(fmin, f.min())
        fmax = max(fmax, f.max())
        done += n
    assert b.lo[0] <= fmin and fmax <= b.hi[0]


@pytest.mark.parametrize("cfg", [0, 1])
def test_point_box_is_point_evaluation(cases, cfg):
    """A zero-radius box reduces IBP to evaluating f, checked against a brute-force
    evaluation that re-solves the base and every outaged network."""
    c = cases(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(9)
    for _ in range(3 if cfg == 0 else 1):
        x = c.box_lo[0] + rng.random(c.n_dev) * (c.box_hi[0] - c.box_lo[0])
        b = O.bound(c, s, lo=x[None], hi=x[None])
        ref = objective_brute(c, x)
        assert abs(b.hi[0] - ref) <= 1e-9 * abs(ref)
        assert abs(b.lo[0] - ref) <= 1e-9 * abs(ref)


def _lp_optimum(c, s, duals: bool = False):
    """max f over the box as an LP (Problem 1 with slacks), scipy HiGHS.
    With duals=True also returns the multipliers of the penalty rows mapped to
    the slopes of oracle.linear_bound: (a_base, a_ctg, a_inj)."""
    sp = pytest.importorskip("scipy.optimize")
    scsp = pytest.importorskip("scipy.sparse")
    ng, nd, nl, nc, nb = c.n_gen, c.n_load, c.n_line, c.n_ctg, c.n_bus
    # variables: x (ng+nd), t_g (ng), t_d (nd), s_inj (nb), s_fb (nl), s_fc (nc*nl)
    nx = ng + nd
    off_tg, off_td = nx, nx + ng
    off_si = off_td + nd
    off_fb = off_si + nb
    off_fc = off_fb + nl
    nv = off_fc + nc * nl
    cost = np.zeros(nv)  # minimise -f
    cost[off_tg:off_tg + ng] = 1.0
    cost[off_td:off_td + nd] = -1.0
    cost[off_si:off_si + nb] = c.zeta_inj
    cost[off_fb:off_fc] = c.zeta_f
    cost[off_fc:] = c.zeta_f
    Nmat = np.zeros((nb, nx))
    Nmat[c.gen_bus, np.arange(ng)] = 1
    Nmat[c.load_bus, ng + np.arange(nd)] = -1
    rows, cols, vals, rhs = [], [], [], []
    W = O.imbalance_matrix(c, s.phi) @ Nmat
    F = s.phi @ Nmat

    def add(coef_x, extra, b):
        r = len(rhs)
        nzx = np.flatnonzero(coef_x)
        rows.extend([r] * nzx.size)
        cols.extend(nzx.tolist())
        vals.extend(coef_x[nzx].tolist())
        for idx, v in extra:
            rows.append(r)
            cols.append(idx)
            vals.append(v)
        rhs.append(b)
    for i in range(nb):
        add(W[i], [(off_si + i, -1)], 0.0)
        add(-W[i], [(off_si + i, -1)], 0.0)
    rc = c.rating
    for l in range(nl):
        add(F[l], [(off_fb + l, -1)], rc[l])
        add(-F[l], [(off_fb + l, -1)], rc[l])
    for k in range(nc):
        Hk = F + np.outer(s.lodf[:, k], F[c.ctg_line[k]])
        for l in range(nl):
            add(Hk[l], [(off_fc + k * nl + l, -1)], rc[l])
            add(-Hk[l], [(off_fc + k * nl + l, -1)], rc[l])
    # PWL epigraphs: convex cost t_g >= piece_i(x), concave value t_d <= piece_i(x)
    def pieces(nseg, a, bk):
        ptr = np.concatenate([[0], np.cumsum(nseg)])
        out = []
        for i in range(len(nseg)):
            aa, bb = a[ptr[i]:ptr[i + 1]], bk[ptr[i]:ptr[i + 1]]
            U = 0.0
            pcs = []
            for m in range(len(aa)):
                pcs.append((aa[m], U - aa[m] * bb[m]))  # value = U_{m-1} + a_m (x - b_m)
                if m + 1 < len(aa):
                    U += aa[m] * (bb[m + 1] - bb[m])
            out.append(pcs)
        return out
    for i, pcs in enumerate(pieces(c.gen_nseg, c.gen_slope, c.gen_bkpt)):
        for (sl, ic) in pcs:
            e = np.zeros(nx)
            e[i] = sl
            add(e, [(off_tg + i, -1)], -ic)
    for j, pcs in enumerate(pieces(c.load_nseg, c.load_slope, c.load_bkpt)):
        for (sl, ic) in pcs:
            e = np.zeros(nx)
            e[ng + j] = -sl
            add(e, [(off_td + j, 1)], ic)
    A = scsp.csr_matrix((vals, (rows, cols)), shape=(len(rhs), nv))
    bounds = [(c.box_lo[0, i], c.box_hi[0, i]) for i in range(nx)] + [(None, None)] * (ng + nd) \
        + [(0, None)] * (nb + nl + nc * nl)
    res = sp.linprog(cost, A_ub=A, b_ub=np.array(rhs), bounds=bounds, method="highs")
    assert res.status == 0, res.message
    if not duals:
        return -res.fun, res.x[:nx]
    # rows: 2 per bus (imbalance), 2 per line (base), 2 per pair (contingency),
    # each pair (+y, -y); the multipliers lam = -marginal >= 0 of y - s <= R
    # and -y - s <= R give the slope a = (lam+ - lam-) / zeta
    lam = -res.ineqlin.marginals
    r = 0
    ib = lam[:2 * nb].reshape(nb, 2)
    r += 2 * nb
    # the imbalance row at the slack is -(1^T p): its slope is minus its multiplier difference
    a_inj = -(ib[c.slack, 0] - ib[c.slack, 1]) / c.zeta_inj
    bb = lam[r:r + 2 * nl].reshape(nl, 2)
    r += 2 * nl
    a_base = (bb[:, 0] - bb[:, 1]) / c.zeta_f
    cc = lam[r:r + 2 * nc * nl].reshape(nc, nl, 2)
    a_ctg = (cc[..., 0] - cc[..., 1]) / c.zeta_f
    return -res.fun, res.x[:nx], (a_base, a_ctg, a_inj)


@pytest.mark.parametrize("cfg,nseg", [(0, 1), (0, 3), (1, 1)])
def test_upper_bound_above_lp_optimum(cfg, nseg):
    c = make_config(cfg, n_seg=nseg)
    s = O.sensitivities(c)
    b = O.bound(c, s)
    opt, xopt = _lp_optimum(c, s)
    # the LP optimum is attained in the box and equals f there
    assert abs(O.objective_point(c, s, xopt) - opt) <= 1e-6 * max(1.0, abs(opt))
    assert b.hi[0] >= opt - 1e-7 * abs(opt)
    gap = abs(b.hi[0] - opt) / abs(opt)
    print(f"cfg{cfg} nseg={nseg}: IBP hi={b.hi[0]:.6g} LP opt={opt:.6g} gap={gap:.3%}")


def test_penalty_map_case_table():
    # (lo, hi, rating) -> (s_lo, s_hi), |x| then max(. - rating, 0)
    table = [
        ((2.0, 5.0, 1.0), (1.0, 4.0)),    # right of zero
        ((-5.0, -2.0, 1.0), (1.0, 4.0)),  # left of zero
        ((-3.0, 5.0, 1.0), (0.0, 4.0)),   # straddles zero, upper side wider
        ((-6.0, 2.0, 1.0), (0.0, 5.0)),   # straddles zero, lower side wider
        ((2.0, 5.0, 6.0), (0.0, 0.0)),    # never violated
        ((2.0, 5.0, 2.0), (0.0, 3.0)),    # tie at the lower end gives 0
        ((0.0, 0.0, 0.0), (0.0, 0.0)),
    ]
    for (lo, hi, rt), (elo, ehi) in table:
        slo, shi = O.viol_interval(lo, hi, rt)
        assert (float(slo), float(shi)) == (elo, ehi)


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_imbalance_closed_form(cases, cfg):
    """(E^T Phi - I) p = -(1^T p) e_slack: the explicit-matrix IBP equals
    |sum c| -/+ sum r at the slack (reading C5)."""
    c = cases(cfg)
    s = O.sensitivities(c)
    cb, rb = O.bus_box(c, c.box_lo, c.box_hi)
    lo, hi = O.imbalance_interval(c, s.phi, cb, rb)
    tc, tr = cb.sum(axis=1), rb.sum(axis=1)
    elo = np.maximum(np.abs(tc) - tr, 0)
    ehi = np.abs(tc) + tr
    scale = np.abs(tc) + tr
    assert np.all(np.abs(lo - elo) <= 1e-9 * scale)
    assert np.all(np.abs(hi - ehi) <= 1e-9 * scale)


def test_relu_chain_matches_direct_pwl():
    rng = np.random.default_rng(4)
    for _ in range(200):
        n = int(rng.integers(1, 5))
        a = rng.uniform(0, 100, n)
        b = np.sort(rng.uniform(0, 300, n))
        b[0] = 0.0
        x1, x2 = np.sort(rng.uniform(0, 400, 2))
        lo, hi = O.relu_chain_interval(a, b, x1, x2)
        assert abs(lo - pwl_direct(a, b, x1)) <= 1e-9 * (1 + abs(lo))
        assert abs(hi - pwl_direct(a, b, x2)) <= 1e-9 * (1 + abs(hi))


def test_tight_inside_paper_mode(cases):
    for cfg in (0, 1):
        c = cases(cfg)
        s = O.sensitivities(c)
        cb, rb = O.bus_box(c, c.box_lo, c.box_hi)
        cent, rad = O.all_ctg_flows(c, s, cb, rb)
        pc, pr = O.paper_mode_flows(c, s, cb, rb)
        tol = 1e-9 * (np.abs(pc) + pr + 1)
        assert np.all(cent - rad >= pc - pr - tol)
        assert np.all(cent + rad <= pc + pr + tol)
        # identical centres, paper radius R_l + |L_lk| R_k
        np.testing.assert_allclose(cent, pc, atol=1e-9 * np.abs(pc).max())


def test_screen_keeps_every_violating_line(cases):
    """A line the paper-mode screen drops has the tight violation interval
    [0, 0] for every contingency (checked against the tight flows summed by
    the plain definition), and dropping those lines leaves the contingency
    penalty sums of the bound unchanged."""
    for cfg, nb in ((0, 1), (1, 1), (1, 4)):
        c = cases(cfg)
        s = O.sensitivities(c)
        if nb > 1:
            rng = np.random.default_rng(5)
            lo, hi = split_boxes(c.box_lo[0], c.box_hi[0], 2, rng)
        else:
            lo, hi = c.box_lo, c.box_hi
        cb, rb = O.bus_box(c, lo, hi)
        live = O.screen_lines(c, s, cb, rb)
        cent, rad = O.all_ctg_flows(c, s, cb, rb)
        viol_hi = np.maximum(np.abs(cent) + rad - c.rating[None, None, :], 0.0)
        assert np.all(viol_hi[:, :, ~live] == 0.0)
        fc_lo, fc_hi = O.ctg_terms(c, s, cb, rb)[:2]
        viol_lo = np.maximum(np.maximum(np.abs(cent) - rad, 0.0) - c.rating[None, None, :], 0.0)
        np.testing.assert_allclose(viol_hi[:, :, live].sum(axis=(1, 2)), fc_hi, rtol=1e-9)
        np.testing.assert_allclose(viol_lo[:, :, live].sum(axis=(1, 2)), fc_lo, rtol=1e-9,
                                   atol=1e-9 * (1 + np.abs(fc_hi).max()))
    # at a point box both radii vanish: the screen keeps exactly the lines
    # with a post-contingency flow above the rating
    c = cases(1)
    s = O.sensitivities(c)
    mid = 0.5 * (c.box_lo + c.box_hi)
    cb, rb = O.bus_box(c, mid, mid)
    cent, _ = O.all_ctg_flows(c, s, cb, rb)
    want = np.any(np.abs(cent[0]) > c.rating[None, :], axis=0)
    np.testing.assert_array_equal(O.screen_lines(c, s, cb, rb), want)
    assert 0 < want.sum() < c.n_line


def test_paper_mode_bound_encloses_tight_and_meets_it_at_points(cases):
    """The paper-mode objective interval contains the tight one (its flow
    radii are larger), and at a point box both radii vanish so the two bounds
    coincide."""
    for cfg in (0, 1):
        c = cases(cfg)
        s = O.sensitivities(c)
        tight = O.bound(c, s)
        paper = O.bound(c, s, mode="paper")
        scale = np.abs(tight.terms["costs"]).sum() + 1e3 * tight.terms["fc"][1].sum()
        assert np.all(paper.hi >= tight.hi - 1e-9 * scale)
        assert np.all(paper.lo <= tight.lo + 1e-9 * scale)
        mid = 0.5 * (c.box_lo + c.box_hi)
        tp = O.bound(c, s, lo=mid, hi=mid)
        pp = O.bound(c, s, lo=mid, hi=mid, mode="paper")
        np.testing.assert_allclose(pp.hi, tp.hi, rtol=1e-9)
        np.testing.assert_allclose(pp.lo, tp.lo, rtol=1e-9)
    # the root box of the 118-bus case: paper mode is strictly looser
    assert paper.hi[0] > tight.hi[0]


def test_inclusion_monotone(cases):
    c = cases(1)
    s = O.sensitivities(c)
    parent = O.bound(c, s)
    rng = np.random.default_rng(2)
    lo, hi = split_boxes(c.box_lo[0], c.box_hi[0], 3, rng)
    child = O.bound(c, s, lo=lo, hi=hi)
    assert np.all(child.hi <= parent.hi[0] + 1e-9 * abs(parent.hi[0]))
    assert np.all(child.lo >= parent.lo[0] - 1e-9 * abs(parent.lo[0]))


def _kink_free_step(c, s, lo, hi):
    """Largest FD step that crosses no kink of hi (|.|, max(.,0)) around the box."""
    cb, rb = O.bus_box(c, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(c, s, cb, rb)
    m = np.abs(np.abs(cent[0]) - rad[0] - c.rating[None, :])
    fb = (cb @ s.phi.T)[0]
    fr = (rb @ np.abs(s.phi).T)[0]
    mb = np.abs(np.abs(fb) - fr - c.rating)
    mi = abs(abs(cb.sum()) - rb.sum())
    # |.| only matters where max(|c| - r - rating, 0) is active, and there c != 0
    dist = min(m.min(), mb.min(), mi)
    hmax = np.abs(s.phi).max() * (1 + np.abs(s.lodf).max())
    return dist / (20 * max(hmax, 1.0))


@pytest.mark.parametrize("cfg", [0, 1])
def test_hand_adjoint_matches_finite_differences(cases, cfg):
    c = cases(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(21 + cfg)
    # a random sub-box so that some contingency violations are certainly active
    lo0, hi0 = c.box_lo[0], c.box_hi[0]
    a = lo0 + 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    b = hi0 - 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    h = _kink_free_step(c, s, a, b)
    assert h > 1e-9
    g_lo, g_hi, _ = O.grad_hi(c, s, lo=a[None], hi=b[None])
    dims = range(c.n_dev) if c.n_dev <= 10 else rng.choice(c.n_dev, 12, replace=False)
    for d in dims:
        for which, g in (("lo", g_lo), ("hi", g_hi)):
            ap, bp, am, bm = a.copy(), b.copy(), a.copy(), b.copy()
            if which == "lo":
                ap[d] += h
                am[d] -= h
            else:
                bp[d] += h
                bm[d] -= h
            fp = O.bound(c, s, lo=ap[None], hi=bp[None]).hi[0]
            fm = O.bound(c, s, lo=am[None], hi=bm[None]).hi[0]
            fd = (fp - fm) / (2 * h)
            scale = max(abs(fd), abs(g[0, d]), 1e-3 * np.abs(g).max())
            assert abs(fd - g[0, d]) <= 1e-4 * scale, (which, d, fd, g[0, d])


def _rating_fd(c, s, lo, hi, field, l, h):
    """Central difference of the oracle's hi in one line's rating.  field is
    "rating" (base ratings; contingency ratings follow when the case has none
    of its own) or "rating_ctg"."""
    import dataclasses
    vals = []
    for sgn in (1.0, -1.0):
        v = getattr(c, field).copy()
        v[l] += sgn * h
        cc = dataclasses.replace(c, **{field: v})
        vals.append(O.bound(cc, s, lo=lo[None], hi=hi[None]).hi[0])
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("cfg", [0, 1])
def test_rating_gradient_matches_finite_differences(cases, cfg):
    """The rating part of the hand adjoint against central differences of the
    oracle's own upper bound, in the shared rating vector, in the base ratings
    alone and in separate contingency ratings.  Each checked line sits at
    least 50 steps from every kink of its violation terms, so the difference
    is exact up to rounding; lines with active pairs are among those checked."""
    import dataclasses
    c = cases(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(31 + cfg)
    lo0, hi0 = c.box_lo[0], c.box_hi[0]
    a = lo0 + 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    b = hi0 - 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    cb, rb = O.bus_box(c, a[None], b[None])
    cent, rad = O.all_ctg_flows(c, s, cb, rb)
    fb, fr = (cb @ s.phi.T)[0], (rb @ np.abs(s.phi).T)[0]
    # the distance of each line's decisions from their kinks
    kc = np.abs(np.abs(cent[0]) - rad[0] - c.rating[None, :]).min(axis=0)
    kb = np.abs(np.abs(fb) - fr - c.rating)
    dist = np.minimum(kc, kb)
    g_base, g_ctg = O.grad_hi_ratings(c, s, a[None], b[None])
    _, _, g_shared = O.grad_hi(c, s, lo=a[None], hi=b[None])
    np.testing.assert_array_equal(g_shared, g_base + g_ctg)
    active = np.flatnonzero((g_base[0] + g_ctg[0]) > 0)
    assert active.size > 0, "the sub-box has no active pair"
    h = 1e-3
    ok = np.flatnonzero(dist > 50 * h)
    lines = np.union1d(np.intersect1d(active, ok)[:6], ok[:3])
    assert np.intersect1d(lines, active).size > 0
    sep = dataclasses.replace(c, rating_ctg=c.rating.copy())
    for l in lines:
        fd = _rating_fd(c, s, a, b, "rating", l, h)
        assert abs(fd - g_shared[0, l]) <= 1e-6 * max(1.0, abs(fd)), (l, fd, g_shared[0, l])
        # with separate contingency ratings, each vector has its own part
        fd_b = _rating_fd(sep, s, a, b, "rating", l, h)
        fd_c = _rating_fd(sep, s, a, b, "rating_ctg", l, h)
        assert abs(fd_b - g_base[0, l]) <= 1e-6 * max(1.0, abs(fd_b)), (l, fd_b, g_base[0, l])
        assert abs(fd_c - g_ctg[0, l]) <= 1e-6 * max(1.0, abs(fd_c)), (l, fd_c, g_ctg[0, l])


def _kink_free_step_lo(c, s, lo, hi):
    """Largest FD step that crosses no kink of lo: |c| + r - rating = 0 for any
    pair or base line, c = 0 for an active one, and sum c = 0 (imbalance)."""
    cb, rb = O.bus_box(c, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(c, s, cb, rb)
    m = np.abs(np.abs(cent[0]) + rad[0] - c.rating[None, :])
    act = (np.abs(cent[0]) + rad[0] - c.rating[None, :]) > 0
    mc = np.abs(cent[0])[act]
    fb = (cb @ s.phi.T)[0]
    fr = (rb @ np.abs(s.phi).T)[0]
    mb = np.abs(np.abs(fb) + fr - c.rating)
    actb = (np.abs(fb) + fr - c.rating) > 0
    dist = min(m.min(), mb.min(), mc.min() if mc.size else np.inf,
               np.abs(fb)[actb].min() if actb.any() else np.inf, abs(cb.sum()))
    hmax = np.abs(s.phi).max() * (1 + np.abs(s.lodf).max())
    return dist / (20 * max(hmax, 1.0))


@pytest.mark.parametrize("cfg", [0, 1])
def test_lower_adjoint_matches_finite_differences(cases, cfg):
    """The hand adjoint of the lower bound (grad_lo) against central
    differences of the oracle's own obj_lo, in box endpoints and ratings."""
    import dataclasses
    c = cases(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(41 + cfg)
    lo0, hi0 = c.box_lo[0], c.box_hi[0]
    a = lo0 + 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    b = hi0 - 0.4 * rng.random(c.n_dev) * (hi0 - lo0)
    h = _kink_free_step_lo(c, s, a, b)
    assert h > 1e-9
    g_lo, g_hi, g_rat = O.grad_lo(c, s, lo=a[None], hi=b[None])
    dims = range(c.n_dev) if c.n_dev <= 10 else rng.choice(c.n_dev, 12, replace=False)
    for d in dims:
        for which, g in (("lo", g_lo), ("hi", g_hi)):
            ap, bp, am, bm = a.copy(), b.copy(), a.copy(), b.copy()
            if which == "lo":
                ap[d] += h
                am[d] -= h
            else:
                bp[d] += h
                bm[d] -= h
            fp = O.bound(c, s, lo=ap[None], hi=bp[None]).lo[0]
            fm = O.bound(c, s, lo=am[None], hi=bm[None]).lo[0]
            fd = (fp - fm) / (2 * h)
            scale = max(abs(fd), abs(g[0, d]), 1e-3 * np.abs(g).max())
            assert abs(fd - g[0, d]) <= 1e-4 * scale, (which, d, fd, g[0, d])
    # ratings: lines whose decisions sit away from their kinks
    cb, rb = O.bus_box(c, a[None], b[None])
    cent, rad = O.all_ctg_flows(c, s, cb, rb)
    fb, fr = (cb @ s.phi.T)[0], (rb @ np.abs(s.phi).T)[0]
    dist = np.minimum(np.abs(np.abs(cent[0]) + rad[0] - c.rating[None, :]).min(axis=0),
                      np.abs(np.abs(fb) + fr - c.rating))
    hr = 1e-3
    lines = np.flatnonzero(dist > 50 * hr)
    active = lines[g_rat[0, lines] > 0]
    pick = np.union1d(active[:6], lines[:2])
    assert active.size > 0
    for l in pick:
        vals = []
        for sg in (1.0, -1.0):
            r = c.rating.copy()
            r[l] += sg * hr
            vals.append(O.bound(dataclasses.replace(c, rating=r), s, lo=a[None], hi=b[None]).lo[0])
        fd = (vals[0] - vals[1]) / (2 * hr)
        assert abs(fd - g_rat[0, l]) <= 1e-6 * max(1.0, abs(fd)), (l, fd, g_rat[0, l])
