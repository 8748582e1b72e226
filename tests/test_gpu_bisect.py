"""Gradient-guided bisection: certified sandwich LB <= max f <= UB against an
LP optimum (scipy HiGHS), monotone bounds, batched and per-box drivers, and
checkpoint/resume of the frontier."""
import os

import numpy as np
import pytest

import oracle as O
from gen import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    return pkg


def test_bisection_sandwich_and_checkpoint(P, tmp_path):
    from paper_2511_15624_gb300.bisect import Bisection
    from tests.test_oracle_ibp import _lp_optimum
    case = make_config(1)
    opt, _ = _lp_optimum(case, O.sensitivities(case))
    gpu = P.Case(case, device=0)
    hist = {}
    for batched in (True, False):
        b = Bisection(gpu, case.box_lo, case.box_hi, max_leaves=64, batched=batched)
        h = b.run(6)
        ubs = [r.ub for r in h]
        lbs = [r.lb for r in h]
        assert all(x >= y for x, y in zip(ubs, ubs[1:])), ubs
        assert all(x <= y for x, y in zip(lbs, lbs[1:])), lbs
        assert lbs[-1] <= opt * (1 - 1e-9 * np.sign(opt)) + 1e-6 * abs(opt)
        assert ubs[-1] >= opt - 1e-6 * abs(opt)
        assert ubs[-1] < ubs[0]  # bisection tightens the root bound
        hist[batched] = h
    # both drivers tighten the bound to the same order
    assert abs(hist[True][-1].ub - hist[False][-1].ub) <= 0.05 * abs(hist[True][0].ub - opt)
    # checkpoint / resume reproduces the frontier
    b = Bisection(gpu, case.box_lo, case.box_hi, max_leaves=64)
    b.run(3)
    path = os.path.join(tmp_path, "frontier.npz")
    b.save(path)
    c = Bisection.load(gpu, path, max_leaves=64)
    assert c.round == 3 and c.ub == b.ub and c.lb == b.lb
    assert np.array_equal(c.lo.cpu().numpy(), b.lo.cpu().numpy())
    r1, r2 = b.step(), c.step()
    assert r1.ub == r2.ub and r1.lb == r2.lb
