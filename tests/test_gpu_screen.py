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


def _check_live_set(case, sens, lo, hi, n, lines):
    cb, rb = O.bus_box(case, lo, hi)
    assert n == len(lines) and np.all(np.diff(lines) > 0)
    kept = np.zeros(case.n_line, bool)
    kept[lines] = True
    must = _tight_live(case, sens, cb, rb)
    assert np.all(kept[must]), np.flatnonzero(must & ~kept)[:10]
    may = O.screen_lines(case, sens, cb, rb, rel=1e-4)
    assert np.all(may[kept]), np.flatnonzero(kept & ~may)[:10]


def _screened_and_plain(P, gpu, lo, hi):
    gpu.set_screen(True)
    s = gpu.bound(lo, hi)
    n, lines = gpu.last_live()
    gpu.set_screen(False)
    p = gpu.bound(lo, hi)
    assert gpu.last_live() == (-1, None)
    gpu.set_screen(True)
    return s, p, n, lines


@pytest.mark.parametrize("cfg", [1, 2])
def test_screen_one_box(P, cfg):
    case = make_config(cfg)
    sens = _sens(cfg, case)
    gpu = P.Case(case, device=0)
    (lo, hi, err), (plo, phi, perr), n, lines = _screened_and_plain(P, gpu, case.box_lo, case.box_hi)
    assert 0 < n <= case.n_line
    _check_live_set(case, sens, case.box_lo, case.box_hi, n, lines)
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
    _check_live_set(case, sens, lo, hi, n, lines)
    assert n < case.n_line
    check_objective(slo, shi, serr, O.bound(case, sens, lo=lo, hi=hi))


def test_screen_multi_box(P):
    case = time_index_boxes(make_config(1), 20, seed=9)
    sens = _sens(1, make_config(1))
    gpu = P.Case(case, device=0)
    (lo, hi, err), (plo, phi, perr), n, lines = _screened_and_plain(P, gpu, case.box_lo, case.box_hi)
    _check_live_set(case, sens, case.box_lo, case.box_hi, n, lines)
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
