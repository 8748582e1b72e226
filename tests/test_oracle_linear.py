"""Pins of the oracle's linear relaxation bound (oracle.linear_bound, the dual
function of the LP whose optimum is max f).

* weak duality: for any slopes in [-1, 1] the bound lies above f at every
  vertex of the 5-bus box, at random points of the 118-bus box, and above the
  LP optimum (scipy HiGHS);
* strong duality: at the LP's own multipliers (mapped to slopes) the bound
  equals the LP optimum;
* the factored line weights give the same value as forming every H_k;
* the readings behind them: f is concave on the box (midpoint inequality on
  random segments, also with 3-segment cost curves), and the LP's optimal
  point attains the LP optimum under the plain point evaluation of f, so the
  LP models max f exactly."""
import itertools

import numpy as np
import pytest

import oracle as O
from gen import make_config
from tests.test_oracle_ibp import _lp_optimum


_LP = {}


def _lp(cfg, nseg, c, s):
    """(optimum, optimal point, slopes from the multipliers), one HiGHS solve
    per configuration for the whole module."""
    key = (cfg, nseg)
    if key not in _LP:
        _LP[key] = _lp_optimum(c, s, duals=True)
    return _LP[key]


def _random_slopes(c, rng, density=0.3):
    a_b = rng.uniform(-1, 1, c.n_line) * (rng.random(c.n_line) < density)
    a_c = rng.uniform(-1, 1, (c.n_ctg, c.n_line)) * (rng.random((c.n_ctg, c.n_line)) < density)
    return a_b, a_c, float(rng.uniform(-1, 1))


@pytest.mark.parametrize("cfg", [0, 1])
def test_weak_duality_for_any_slopes(cfg):
    c = make_config(cfg)
    s = O.sensitivities(c)
    opt = _lp(cfg, 1, c, s)[0]
    rng = np.random.default_rng(5 + cfg)
    lo, hi = c.box_lo[0], c.box_hi[0]
    if cfg == 0:
        pts = [np.where(np.array(bits, bool), hi, lo) for bits in itertools.product((0, 1), repeat=c.n_dev)]
    else:
        pts = [lo + rng.random(c.n_dev) * (hi - lo) for _ in range(300)]
    fvals = np.array([O.objective_point(c, s, x) for x in pts])
    for trial in range(4):
        a_b, a_c, a0 = _random_slopes(c, rng, density=[1.0, 0.3, 0.05, 0.0][trial])
        u = O.linear_bound(c, s, lo, hi, a_b, a_c, a0)
        assert u >= fvals.max() - 1e-9 * abs(u), (trial, u, fvals.max())
        assert u >= opt - 1e-9 * abs(opt), (trial, u, opt)


@pytest.mark.parametrize("cfg", [0, 1])
def test_strong_duality_at_the_lp_multipliers(cfg):
    c = make_config(cfg)
    s = O.sensitivities(c)
    opt, _, (a_b, a_c, a0) = _lp(cfg, 1, c, s)
    assert np.all(np.abs(a_b) <= 1 + 1e-9) and np.all(np.abs(a_c) <= 1 + 1e-9) and abs(a0) <= 1 + 1e-9
    u = O.linear_bound(c, s, c.box_lo[0], c.box_hi[0], np.clip(a_b, -1, 1), np.clip(a_c, -1, 1),
                       float(np.clip(a0, -1, 1)))
    print(f"cfg {cfg}: LP optimum {opt:.9g}, linear bound at its multipliers {u:.9g}")
    assert abs(u - opt) <= 1e-6 * abs(opt), (u, opt)


@pytest.mark.parametrize("cfg", [0, 1])
def test_factored_weights_equal_explicit_rows(cfg):
    c = make_config(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(9)
    a_b, a_c, a0 = _random_slopes(c, rng, 0.5)
    u1 = O.linear_bound(c, s, c.box_lo[0], c.box_hi[0], a_b, a_c, a0)
    u2 = O.linear_bound(c, s, c.box_lo[0], c.box_hi[0], a_b, a_c, a0, factored=True)
    assert abs(u1 - u2) <= 1e-10 * max(1.0, abs(u1))


@pytest.mark.parametrize("cfg,nseg", [(0, 1), (0, 3), (1, 1)])
def test_objective_is_concave(cfg, nseg):
    """f((x + y) / 2) >= (f(x) + f(y)) / 2 on random segments of the box."""
    c = make_config(cfg, n_seg=nseg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(7 + cfg + nseg)
    lo, hi = c.box_lo[0], c.box_hi[0]
    worst = np.inf
    for _ in range(200):
        x = lo + rng.random(c.n_dev) * (hi - lo)
        y = lo + rng.random(c.n_dev) * (hi - lo)
        fx, fy = O.objective_point(c, s, x), O.objective_point(c, s, y)
        fm = O.objective_point(c, s, 0.5 * (x + y))
        scale = max(abs(fx), abs(fy), 1.0)
        worst = min(worst, (fm - 0.5 * (fx + fy)) / scale)
    assert worst >= -1e-12, worst


@pytest.mark.parametrize("cfg,nseg", [(0, 1), (0, 3), (1, 1)])
def test_lp_point_attains_the_lp_optimum(cfg, nseg):
    """The LP's optimal dispatch, evaluated by the plain point evaluation of
    f (every outaged network's flows), gives the LP optimum."""
    c = make_config(cfg, n_seg=nseg)
    s = O.sensitivities(c)
    opt, x, _ = _lp(cfg, nseg, c, s)
    f = O.objective_point(c, s, x)
    assert abs(f - opt) <= 1e-6 * max(abs(opt), 1.0), (f, opt)
