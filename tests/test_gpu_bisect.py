"""Gradient-guided bisection: certified sandwich LB <= max f <= UB against an
LP optimum (scipy HiGHS), monotone bounds, batched and per-box drivers, and
checkpoint/resume of the frontier; with IBP leaves the gap to the optimum
shrinks by a stated fraction, and with linear-relaxation leaves the sandwich
closes to within 0.25% of the optimum on the 118-bus box."""
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


def test_ibp_leaves_alone_barely_move_the_bound(P):
    """On the 118-bus box, 12 rounds of IBP leaves (the frontier filled to 256
    leaves after 8 rounds) lower UB, but only by a small fraction of its excess
    over the optimum (measured: 0.15%): f is concave, its IBP looseness comes
    from the same devices entering many penalty terms, and splitting one
    coordinate of a 153-dimensional box at a time does not remove it.  The
    linear leaves of the next test close the gap instead."""
    from paper_2511_15624_gb300.bisect import Bisection
    from tests.test_oracle_ibp import _lp_optimum
    case = make_config(1)
    opt, _ = _lp_optimum(case, O.sensitivities(case))
    gpu = P.Case(case, device=0)
    h = Bisection(gpu, case.box_lo, case.box_hi, max_leaves=256).run(12)
    gpu.close()
    ex0, ex = h[0].ub - opt, h[-1].ub - opt
    print(f"excess UB - opt: root {ex0:.6g}, after {len(h)} rounds {ex:.6g} "
          f"({h[-1].n_leaves} leaves); LB {h[-1].lb:.9g} opt {opt:.9g}")
    assert h[-1].n_leaves == 256
    assert -1e-6 * abs(opt) <= ex < ex0
    assert h[-1].lb <= opt + 1e-6 * abs(opt)


@pytest.mark.parametrize("batched", [True, False])
def test_linear_bisection_closes_the_sandwich(P, batched):
    """Linear-relaxation leaves (children continue their parent's slopes):
    after 4 rounds of up to 8 leaves, opt - 0.25% <= LB <= opt <= UB <=
    opt + 0.25%, i.e. at least 99.7% of the IBP root bound's excess over opt
    removed (measured: UB 0.04% above opt, LB 0.01% below)."""
    from paper_2511_15624_gb300.bisect import Bisection
    from tests.test_oracle_ibp import _lp_optimum
    case = make_config(1)
    opt, _ = _lp_optimum(case, O.sensitivities(case))
    gpu = P.Case(case, device=0)
    b = Bisection(gpu, case.box_lo, case.box_hi, max_leaves=8, batched=batched, bound="linear",
                  linear_iters=2000, linear_root_iters=20000)
    h = b.run(4)
    for r in h:
        print(f"round {r.round}: UB {r.ub:.9g} LB {r.lb:.9g} gap {r.gap:.3e} leaves {r.n_leaves} "
              f"{r.round_seconds:.3f} s ({r.bound_seconds:.3f} s in bounds)")
    ibp_root = float(gpu.bound(case.box_lo, case.box_hi)[1][0])
    tol = 1e-6 * abs(opt)
    assert h[-1].ub - opt <= 0.003 * (ibp_root - opt), (h[-1].ub, ibp_root, opt)
    assert all(x >= y for x, y in zip([r.ub for r in h], [r.ub for r in h][1:]))
    assert h[-1].ub >= opt - tol and h[-1].lb <= opt + tol
    assert h[-1].ub <= opt + 0.0025 * abs(opt), (h[-1].ub, opt)
    assert h[-1].lb >= opt - 0.0025 * abs(opt), (h[-1].lb, opt)
    gpu.close()
