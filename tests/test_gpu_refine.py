"""FP64 refinement of the terms that can reach obj_hi (ibp_case_set_refine).

With the refinement on, every base line and contingency pair whose lower
violation bound can be positive is recomputed from the FP64 PTDF with FP64
sums and an explicit error bound, so obj_hi meets the oracle's FP64 value up
to FP64 rounding and the FP64 build allowance, and its error bound shrinks to
the same size.  With it off the FP32 path's own bound holds; the two results
agree within the sum of their error bounds.  Checked for the one-box,
many-box and paper-mode paths, with and without the screen and the network
reduction."""
import numpy as np
import pytest

import oracle as O
from gen import make_config
from gen.cases import make_two_core_case, time_index_boxes
from tests.test_gpu_parity import F64, _sens, check_objective, side_scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    return pkg


def _near_exact(hi, err, ref):
    """obj_hi within FP64 rounding of the oracle: 1e-9 of its own terms."""
    hi_s, _ = side_scales(ref)
    assert np.all(np.abs(hi - ref.hi) <= 1e-9 * hi_s + F64 * hi_s), (hi - ref.hi, hi_s)
    assert np.all(err[:, 0] <= 1e-9 * hi_s), (err[:, 0], hi_s)


@pytest.mark.parametrize("cfg", [1, 2])
def test_refined_hi_is_fp64_exact(P, cfg):
    case = make_config(cfg)
    sens = _sens(cfg, case)
    ref = O.bound(case, sens)
    gpu = P.Case(case, device=0)
    for screen, reduce in ((True, True), (False, False)):
        gpu.set_screen(screen)
        gpu.set_reduction(reduce)
        lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
        check_objective(lo, hi, err, ref)
        _near_exact(hi, err, ref)
    # without the refinement: the FP32 bound, within both error bounds
    gpu.set_refine(False)
    lo0, hi0, err0 = gpu.bound(case.box_lo, case.box_hi)
    assert np.all(hi0 >= ref.hi - F64 * side_scales(ref)[0])
    assert np.all(np.abs(hi0 - hi) <= err0[:, 0] + err[:, 0])
    assert np.all(err0[:, 0] > err[:, 0])
    # obj_lo does not use the refinement
    assert np.array_equal(lo0, lo) or np.all(np.abs(lo0 - lo) <= err0[:, 1] + err[:, 1])


def test_refined_many_boxes_and_paper_mode(P):
    base = make_config(1)
    sens = _sens(1, base)
    case = time_index_boxes(base, 20, seed=9)
    gpu = P.Case(case, device=0)
    ref = O.bound(case, sens)
    lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
    check_objective(lo, hi, err, ref)
    _near_exact(hi, err, ref)
    plo, phi, perr = gpu.bound_paper(case.box_lo, case.box_hi)
    pref = O.bound(case, sens, mode="paper")
    check_objective(plo, phi, perr, pref)
    _near_exact(phi, perr, pref)


def test_refined_bridges_in_closed_form(P):
    """Bridge lines (never contingencies) keep their base flow under every
    outage; the reduced path adds their n_c pairs in closed form, and the
    refinement recomputes those too."""
    case = make_two_core_case()
    sens = O.sensitivities(case)
    ref = O.bound(case, sens)
    gpu = P.Case(case, device=0)
    assert gpu.info().n_bridges > 0
    lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
    check_objective(lo, hi, err, ref, rel_scale=np.abs(ref.terms["costs"]).sum(axis=1))
    _near_exact(hi, err, ref)
