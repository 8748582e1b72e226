"""Pins of the oracle's linear relaxation bound (oracle.linear_bound, the dual
function of the LP whose optimum is max f).

* weak duality: for any slopes in [-1, 1] the bound lies above f at every
  vertex of the 5-bus box, at random points of the 118-bus box, and above the
  LP optimum (scipy HiGHS);
* strong duality: at the LP's own multipliers (mapped to slopes) the bound
  equals the LP optimum;
* the factored line weights give the same value as forming every H_k."""
import itertools

import numpy as np
import pytest

import oracle as O
from gen import make_config
from tests.test_oracle_ibp import _lp_optimum


def _random_slopes(c, rng, density=0.3):
    a_b = rng.uniform(-1, 1, c.n_line) * (rng.random(c.n_line) < density)
    a_c = rng.uniform(-1, 1, (c.n_ctg, c.n_line)) * (rng.random((c.n_ctg, c.n_line)) < density)
    return a_b, a_c, float(rng.uniform(-1, 1))


@pytest.mark.parametrize("cfg", [0, 1])
def test_weak_duality_for_any_slopes(cfg):
    c = make_config(cfg)
    s = O.sensitivities(c)
    opt, _ = _lp_optimum(c, s)
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
    opt, _, (a_b, a_c, a0) = _lp_optimum(c, s, duals=True)
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
