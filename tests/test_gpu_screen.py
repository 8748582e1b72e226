"""Paper-mode line screen on the GPU (calls through the C ABI).

* soundness: every line whose tight contingency interval can exceed its rating
  (oracle, FP64, the plain definition) is kept;
* efficacy: every line that the oracle's paper-mode interval clears with a
  1e-4 relative margin below its rating is dropped;
* the screened bound contains the oracle's and agrees with the unscreened
  one within their error bounds (only the rounding order of the sums moves);
* calls that ask for flows, and a screen switched off, report -1.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from gen import make_config, split_boxes
from gen.cases import time_index_boxes
from tests.test_gpu_parity import _sens, check_objective

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    return pkg


def _tight_live(case, sens, cb, rb):
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    rating = case.rating if case.rating_ctg is None else case.rating_ctg
    return np.any(np.abs(cent) + rad > rating[None, None, :], axis=(0, 1))


def _check_live_set(case, sens, lo, hi, n, lines, bridges=None):
    """bridges: lines the network reduction handles in closed form (never kept)."""
    cb, rb = O.bus_box(case, lo, hi)
    assert n == len(lines) and np.all(np.diff(lines) > 0)
    kept = np.zeros(case.n_line, bool)
    kept[lines] = True
    must = _tight_live(case, sens, cb, rb)
    if bridges is not None:
        assert not np.any(kept & bridges)
        must &= ~bridges
    assert np.all(kept[must]), np.flatnonzero(must & ~kept)[:10]
    may = O.screen_lines(case, sens, cb, rb, rel=1e-4)
    assert np.all(may[kept]), np.flatnonzero(kept & ~may)[:10]


def _screened_and_plain(P, gpu, lo, hi):
    """The default call (screen and network reduction on) and the plain one."""
    gpu.set_screen(True)
    s = gpu.bound(lo, hi)
    n, lines = gpu.last_live()
    gpu.set_screen(False)
    gpu.set_reduction(False)
    p = gpu.bound(lo, hi)
    assert gpu.last_live() == (-1, None)
    gpu.set_screen(True)
    gpu.set_reduction(True)
    return s, p, n, lines


def _bridges(gpu):
    return gpu.reduction()[1].astype(bool)


@pytest.mark.parametrize("cfg", [1, 2])
def test_screen_one_box(P, cfg):
    case = make_config(cfg)
    sens = _sens(cfg, case)
    gpu = P.Case(case, device=0)
    (lo, hi, err), (plo, phi, perr), n, lines = _screened_and_plain(P, gpu, case.box_lo, case.box_hi)
    assert 0 < n <= case.n_line
    _check_live_set(case, sens, case.box_lo, case.box_hi, n, lines, _bridges(gpu))
    ref = O.bound(case, sens)
    check_objective(lo, hi, err, ref)
    check_objective(plo, phi, perr, ref)
    assert np.all(np.abs(hi - phi) <= err[:, 0] + perr[:, 0])
    assert np.all(np.abs(lo - plo) <= err[:, 1] + perr[:, 1])


def test_screen_small_boxes_drop_many_lines(P):
    """Sub-boxes near the dispatch midpoint clear most lines; a ragged live
    count exercises the partial last line tile."""
    case = make_config(2)
    sens = _sens(2, case)
    gpu = P.Case(case, device=0)
    mid = 0.5 * (case.box_lo[0] + case.box_hi[0])
    w = 0.02 * (case.box_hi[0] - case.box_lo[0])
    lo, hi = (mid - w)[None], (mid + w)[None]
    (slo, shi, serr), _, n, lines = _screened_and_plain(P, gpu, lo, hi)
    _check_live_set(case, sens, lo, hi, n, lines, _bridges(gpu))
    assert n < case.n_line
    check_objective(slo, shi, serr, O.bound(case, sens, lo=lo, hi=hi))


def test_screen_multi_box(P):
    case = time_index_boxes(make_config(1), 20, seed=9)
    sens = _sens(1, make_config(1))
    gpu = P.Case(case, device=0)
    (lo, hi, err), (plo, phi, perr), n, lines = _screened_and_plain(P, gpu, case.box_lo, case.box_hi)
    _check_live_set(case, sens, case.box_lo, case.box_hi, n, lines, _bridges(gpu))
    ref = O.bound(case, sens)
    check_objective(lo, hi, err, ref)
    assert np.all(np.abs(hi - phi) <= err[:, 0] + perr[:, 0])


def test_screen_everything_dropped_and_flows_unscreened(P):
    base = make_config(1)
    sens = _sens(1, base)
    big = dataclasses.replace(base, rating_ctg=np.full(base.n_line, 1e9))
    gpu = P.Case(big, device=0)
    lo, hi, err = gpu.bound(big.box_lo, big.box_hi)
    n, lines = gpu.last_live()
    assert n == 0 and lines.size == 0
    check_objective(lo, hi, err, O.bound(big, sens))
    # flows requested: the screen stays off for that call
    gpu2 = P.Case(base, device=0)
    gpu2.bound(base.box_lo, base.box_hi, flows=True)
    assert gpu2.last_live() == (-1, None)


def test_screen_adjoint_unchanged(P):
    case = make_config(1)
    gpu = P.Case(case, device=0)
    rng = np.random.default_rng(4)
    lo, hi = split_boxes(case.box_lo[0], case.box_hi[0], 2, rng)
    g = np.ones(lo.shape[0])
    gpu.set_screen(True)
    a_lo, a_hi, a_r = gpu.backward(lo, hi, g, want_rating=True)
    gpu.set_screen(False)
    b_lo, b_hi, b_r = gpu.backward(lo, hi, g, want_rating=True)
    # same active pairs; only the order of the FP64 atomic sums can differ
    scale = 1e-9 * (1 + np.abs(b_lo).max() + np.abs(b_hi).max())
    np.testing.assert_allclose(a_lo, b_lo, rtol=0, atol=scale)
    np.testing.assert_allclose(a_hi, b_hi, rtol=0, atol=scale)
    np.testing.assert_array_equal(a_r, b_r)


def _modes(P, gpu, lo, hi):
    """Bounds with (screen, reduction) on/off."""
    out = {}
    for screen, reduce in ((True, True), (False, True), (True, False), (False, False)):
        gpu.set_screen(screen)
        gpu.set_reduction(reduce)
        out[(screen, reduce)] = gpu.bound(lo, hi)
    gpu.set_screen(True)
    gpu.set_reduction(True)
    return out


@pytest.mark.parametrize("which", ["cfg2", "two-core", "sparse"])
def test_reduction_one_box(P, which):
    """Exact network reduction (bridges in closed form, bus classes): every
    combination with the line screen contains the oracle's bound and agrees
    with the plain path within the two error bounds."""
    from gen import make_network_case
    from gen.cases import make_two_core_case
    if which == "cfg2":
        case = make_config(2)
        sens = _sens(2, case)
    elif which == "two-core":
        case = make_two_core_case()
        sens = O.sensitivities(case)
    else:
        case = make_network_case("sparse", 160, 175, 30, 70, seed=91)
        sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    info = gpu.info()
    assert info.n_bus_classes < info.n_active and info.n_bridges > 0
    ref = O.bound(case, sens)
    out = _modes(P, gpu, case.box_lo, case.box_hi)
    plo, phi, perr = out[(False, False)]
    # the small networks' objectives cancel to ~10% of their cost terms: the
    # 1e-5 relative bar is taken of the cost scale there
    rs = None if which == "cfg2" else np.abs(ref.terms["costs"]).sum(axis=1)
    for key, (lo, hi, err) in out.items():
        check_objective(lo, hi, err, ref, rel_scale=rs)
        assert np.all(np.abs(hi - phi) <= err[:, 0] + perr[:, 0]), key
        assert np.all(np.abs(lo - plo) <= err[:, 1] + perr[:, 1]), key
    # the reduced call keeps no bridge line for the contingency kernel
    gpu.bound(case.box_lo, case.box_hi)
    n, lines = gpu.last_live()
    _, br = gpu.reduction()
    assert not np.any(br[lines])


def test_reduction_multi_box_and_adjoint(P):
    from gen.cases import make_two_core_case
    base = make_two_core_case()
    sens = O.sensitivities(base)
    rng = np.random.default_rng(12)
    lo, hi = split_boxes(base.box_lo[0], base.box_hi[0], 4, rng)
    case = base.with_boxes(lo, hi)
    gpu = P.Case(case, device=0)
    ref = O.bound(case, sens)
    out = _modes(P, gpu, lo, hi)
    rs = np.abs(ref.terms["costs"]).sum(axis=1)
    for key, (blo, bhi, berr) in out.items():
        check_objective(blo, bhi, berr, ref, rel_scale=rs)
    # the adjoints compare only where no active-set decision sits at its kink
    from tests.test_gpu_adjoint import _kink_free
    keep = [j for j in range(lo.shape[0]) if _kink_free(case, sens, lo[j], hi[j])[0]]
    assert len(keep) >= 4
    lo, hi = lo[keep], hi[keep]
    case = case.with_boxes(lo, hi)
    g = np.ones(lo.shape[0])
    grads = {}
    for reduce in (True, False):
        gpu.set_reduction(reduce)
        grads[reduce] = gpu.backward(lo, hi, g, want_rating=True)
    gpu.set_reduction(True)
    a_lo, a_hi, a_r = grads[True]
    b_lo, b_hi, b_r = grads[False]
    scale = 1e-9 * (1 + np.abs(b_lo).max() + np.abs(b_hi).max())
    np.testing.assert_allclose(a_lo, b_lo, rtol=0, atol=scale)
    np.testing.assert_allclose(a_hi, b_hi, rtol=0, atol=scale)
    np.testing.assert_array_equal(a_r, b_r)
    # and the hand adjoint of the oracle on the same boxes
    o_lo, o_hi, o_r = O.grad_hi(case, sens, lo, hi)
    tol = 1e-6 * (1 + np.abs(o_lo).max() + np.abs(o_hi).max())
    np.testing.assert_allclose(a_lo, o_lo, rtol=0, atol=tol)
    np.testing.assert_allclose(a_hi, o_hi, rtol=0, atol=tol)


@pytest.mark.parametrize("which", ["cfg1", "cfg2", "multi", "point"])
def test_paper_mode_bound(P, which):
    """ibp_bound_paper against the oracle's paper-mode bound (the paper's own
    two-part contingency intervals): sound, within 1e-5 and its own error
    bound; it encloses the tight bound of ibp_bound, and equals it at a point
    box, where both radii vanish."""
    if which == "multi":
        case = time_index_boxes(make_config(1), 20, seed=9)
        sens = _sens(1, make_config(1))
        lo, hi = case.box_lo, case.box_hi
    else:
        cfg = 2 if which == "cfg2" else 1
        case = make_config(cfg)
        sens = _sens(cfg, case)
        lo, hi = case.box_lo, case.box_hi
        if which == "point":
            lo = hi = 0.5 * (case.box_lo + case.box_hi)
    gpu = P.Case(case, device=0)
    plo, phi, perr = gpu.bound_paper(lo, hi)
    ref = O.bound(case, sens, lo=lo, hi=hi, mode="paper")
    check_objective(plo, phi, perr, ref)
    tlo, thi, terr = gpu.bound(lo, hi)
    assert np.all(phi >= thi - terr[:, 0]) and np.all(plo <= tlo + terr[:, 1])
    if which == "point":
        assert np.all(np.abs(phi - thi) <= perr[:, 0] + terr[:, 0])
    else:
        assert np.all(phi > thi)
