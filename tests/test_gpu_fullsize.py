"""Parity at the full 8316-bus size, in the launch configurations bench.py
times: one box with the library defaults (line screen and network reduction
on), and one box out of a 32-box call (multi-box kernel).  The oracle bounds
the same boxes in full (all contingencies x all lines x all buses, about half
a minute on the host cores per box); flow intervals are compared on a sample
of pairs that the oracle computes one by one.  The measured deviations of both
ends are printed and held to the 1e-5 bar: obj_hi may not fall below the
oracle's by more than the FP64 build allowance (1e-10 of its own terms, about
0.1 $ here), and neither end may move by more than 1e-5 of the oracle's
value."""
import numpy as np
import pytest

import oracle as O
from gen import make_config
from gen.cases import time_index_boxes
from tests.test_gpu_parity import F64, check_flows, check_objective, side_scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    case = make_config(3)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    return P, torch, case, sens, gpu


def _report(olo, ohi, err, ref, what):
    dev_hi, dev_lo = check_objective(olo, ohi, err, ref)
    hi_s, lo_s = side_scales(ref)
    print(f"mesh8316 {what}: (hi - oracle) / |oracle| = {dev_hi[0]:+.3e}, "
          f"(lo - oracle) / |oracle| = {dev_lo[0]:+.3e}, err_hi / |hi| = {err[0, 0] / abs(ref.hi[0]):.3e}, "
          f"err_lo / |lo| = {err[0, 1] / abs(ref.lo[0]):.3e}, FP64 allowance hi {F64 * hi_s[0]:.3g} $")
    # sound (up to the FP64 allowance) and within 1e-5 at both ends
    assert dev_hi[0] >= -F64 * hi_s[0] / abs(ref.hi[0]) and dev_hi[0] <= 1e-5
    assert dev_lo[0] <= F64 * lo_s[0] / abs(ref.lo[0]) and dev_lo[0] >= -1e-5


_ROOT = {}


def _root_bound(case, sens):
    """The oracle's complete bound of the root box (computed once per module)."""
    if "ref" not in _ROOT:
        _ROOT["ref"] = O.bound(case, sens)
    return _ROOT["ref"]


def test_fullsize_one_box_default_launch(env):
    P, torch, case, sens, gpu = env
    lo = torch.tensor(case.box_lo, device="cuda")
    hi = torch.tensor(case.box_hi, device="cuda")
    olo, ohi, err = (t.cpu().numpy() for t in gpu.bound(lo, hi))
    n, _ = gpu.last_live()
    assert 0 < n < case.n_line  # the screen and the reduction were in the path
    ref = _root_bound(case, sens)
    _report(olo, ohi, err, ref, "one box")


def test_fullsize_box_of_32_box_call(env):
    P, torch, case, sens, gpu = env
    bcase = time_index_boxes(case, 32, seed=2003)
    lo = torch.tensor(bcase.box_lo, device="cuda")
    hi = torch.tensor(bcase.box_hi, device="cuda")
    olo, ohi, err = (t.cpu().numpy() for t in gpu.bound(lo, hi))
    j = 17
    ref = O.bound(case, sens, lo=bcase.box_lo[j:j + 1], hi=bcase.box_hi[j:j + 1])
    _report(olo[j:j + 1], ohi[j:j + 1], err[j:j + 1], ref, "box 17 of 32")


def test_fullsize_sampled_flows(env):
    P, torch, case, sens, gpu = env
    lo, hi, err, flo, fhi = gpu.bound(case.box_lo, case.box_hi, flows=True)
    rng = np.random.default_rng(83)
    pk = rng.integers(0, case.n_ctg, 20000)
    pl = rng.integers(0, case.n_line, 20000)
    pl[:200] = case.ctg_line[pk[:200]]  # include outaged lines
    check_flows(case, sens, case.box_lo, case.box_hi, flo, fhi, pk, pl)


def test_fullsize_linear_bound_is_certified(env):
    """The linear relaxation at 8316 buses: at the slopes the GPU ends with,
    the oracle's own evaluation of the dual function (factored form, pinned
    against the explicit one on small cases) lies at or below the GPU's
    certified value and within its error bound plus the FP64 build allowance
    (1e-10 of the objective's terms); the bound is far below IBP's."""
    P, torch, case, sens, gpu = env
    ub, err, xp = gpu.bound_linear(case.box_lo, case.box_hi, n_iter=2000)
    a_c, a_b, a0 = gpu.linear_slopes(1)
    val = O.linear_bound(case, sens, case.box_lo[0], case.box_hi[0], a_b[0], a_c[0], a0[0], factored=True)
    ref = _root_bound(case, sens)
    scale = float(np.abs(ref.terms["costs"]).sum() + case.zeta_inj * ref.terms["inj"][1][0]
                  + case.zeta_f * (ref.terms["fb"][1][0] + ref.terms["fc"][1][0]))
    d = F64 * scale
    print(f"mesh8316 linear: GPU {ub[0]:.10g} (err {err[0]:.3g}), oracle at its slopes {val:.10g}, "
          f"difference {ub[0] - val:.3g}, allowance {d:.3g}; IBP hi {ref.hi[0]:.6g}")
    assert ub[0] >= val - d, (ub[0], val, d)
    assert ub[0] - val <= err[0] + d, (ub[0] - val, err[0], d)
    assert ub[0] < ref.hi[0]
