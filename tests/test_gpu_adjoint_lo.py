"""Adjoint of obj_lo (ibp_bound_backward_lo) and the ratings as inputs of the
autograd.Function (ibp_case_set_ratings).

The GPU adjoint of the lower bound is compared with the oracle's hand adjoint
(oracle.grad_lo, itself pinned by finite differences on the host) and with
FP64 central differences of the oracle's obj_lo, 1e-4 relative, on sub-boxes
whose decisions sit away from every kink of obj_lo.  The autograd.Function
with a rating tensor is compared with central differences of the oracle in
the shared ratings, and with the oracle's hand gradients of both ends."""
import dataclasses

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


def _lo_kinks(case, sens, lo, hi):
    """(distance of obj_lo's active-set decisions from their kinks, distance
    of the active flows' centres from 0, flow scale)."""
    cb, rb = O.bus_box(case, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    up = np.abs(cent[0]) + rad[0] - case.rating[None, :]
    fb, fr = (cb @ sens.phi.T)[0], (rb @ np.abs(sens.phi).T)[0]
    upb = np.abs(fb) + fr - case.rating
    d_up = min(np.abs(up).min(), np.abs(upb).min(), abs(cb.sum()))
    d_c = min(np.abs(cent[0])[up > 0].min() if (up > 0).any() else np.inf,
              np.abs(fb)[upb > 0].min() if (upb > 0).any() else np.inf)
    scale = float((np.abs(cent) + rad).max())
    return d_up, d_c, scale


def _lo_kink_free(case, sens, lo, hi):
    """(ok, FD step).  The GPU decides each active set membership from its
    FP32 interval (within about 1e-6 of the flow scale) and each centre's sign
    from its FP32 centre (within about 2.1 u32 of the centre's operands, below
    1e-6 of the flow scale here), so both must clear those margins; the step
    keeps every decision of the oracle fixed."""
    d_up, d_c, scale = _lo_kinks(case, sens, lo, hi)
    hmax = np.abs(sens.phi).max() * (1 + np.abs(sens.lodf).max())
    ok = d_up > 1e-5 * (1 + scale) and d_c > 1e-6 * (1 + scale)
    return ok, min(d_up, d_c) / (20 * max(hmax, 1.0))


def _sub_boxes(case, n, seed, shrink=0.45):
    rng = np.random.default_rng(seed)
    lo0, hi0 = case.box_lo[0], case.box_hi[0]
    a = lo0 + shrink * rng.random((n, case.n_dev)) * (hi0 - lo0)
    b = hi0 - shrink * rng.random((n, case.n_dev)) * (hi0 - lo0)
    return np.minimum(a, b), np.maximum(a, b)


@pytest.mark.parametrize("cfg", [0, 1])
def test_lo_adjoint_matches_oracle_and_fd(P, cfg):
    case = make_config(cfg)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    lo_b, hi_b = _sub_boxes(case, 40, 70 + cfg)
    picked = []
    for j in range(lo_b.shape[0]):
        ok, h = _lo_kink_free(case, sens, lo_b[j], hi_b[j])
        if ok:
            picked.append((j, h))
        if len(picked) == 2:
            break
    assert picked, "no kink-free sub-box drawn"
    for j, h in picked:
        lo, hi = lo_b[j:j + 1], hi_b[j:j + 1]
        glo, ghi, grat = gpu.backward(lo, hi, np.ones(1), want_rating=True, side="lo")
        o_lo, o_hi, o_rat = O.grad_lo(case, sens, lo=lo, hi=hi)
        scale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
        np.testing.assert_allclose(glo, o_lo, rtol=0, atol=1e-4 * scale)
        np.testing.assert_allclose(ghi, o_hi, rtol=0, atol=1e-4 * scale)
        np.testing.assert_allclose(grat, o_rat, rtol=0, atol=1e-9 * max(1.0, np.abs(o_rat).max()))
        rng = np.random.default_rng(200 + j)
        dims = rng.choice(case.n_dev, min(case.n_dev, 6), replace=False)
        for d in dims:
            for which, g in (("lo", glo), ("hi", ghi)):
                ap, bp, am, bm = lo[0].copy(), hi[0].copy(), lo[0].copy(), hi[0].copy()
                if which == "lo":
                    ap[d] += h
                    am[d] -= h
                else:
                    bp[d] += h
                    bm[d] -= h
                fp = O.bound(case, sens, lo=ap[None], hi=bp[None]).lo[0]
                fm = O.bound(case, sens, lo=am[None], hi=bm[None]).lo[0]
                fd = (fp - fm) / (2 * h)
                assert abs(fd - g[0, d]) <= 1e-4 * max(abs(fd), 1e-3 * scale), (which, d, fd, g[0, d])
    gpu.close()


def test_set_ratings_matches_a_new_case(P):
    import torch
    case = make_config(1)
    r2 = case.rating * np.linspace(0.9, 1.1, case.n_line)
    gpu = P.Case(case, device=0)
    gpu.set_ratings(r2)
    lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
    fresh = P.Case(dataclasses.replace(case, rating=r2), device=0)
    lo2, hi2, err2 = fresh.bound(case.box_lo, case.box_hi)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2) and np.array_equal(err, err2)
    # device pointers; a bad entry leaves the ratings unchanged and is reported
    bad = torch.tensor(r2, device="cuda")
    bad[5] = -1.0
    gpu.set_ratings(bad)
    torch.cuda.synchronize()
    with pytest.raises(P.IBPError) as ei:
        gpu.sync()
    assert ei.value.status == P._abi.IBP_EINVAL
    lo3, hi3, _ = (t for t in gpu.bound(torch.tensor(case.box_lo, device="cuda"),
                                        torch.tensor(case.box_hi, device="cuda")))
    torch.cuda.synchronize()
    assert float(hi3[0]) == hi[0] and float(lo3[0]) == lo[0]
    fresh.close()
    gpu.close()


def test_autograd_ratings_and_both_ends(P):
    import torch
    from paper_2511_15624_gb300.autograd import ibp_bound
    case = make_config(1)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    lo_b, hi_b = _sub_boxes(case, 40, 91)
    keep = []
    for j in range(lo_b.shape[0]):
        from tests.test_gpu_adjoint import _kink_free
        if _lo_kink_free(case, sens, lo_b[j], hi_b[j])[0] and _kink_free(case, sens, lo_b[j], hi_b[j])[0]:
            keep.append(j)
        if len(keep) == 3:
            break
    assert len(keep) >= 2
    lo_b, hi_b = lo_b[keep], hi_b[keep]
    nb = len(keep)
    w_hi = np.linspace(1.0, 2.0, nb)
    w_lo = np.linspace(-0.5, 0.5, nb)
    tlo = torch.tensor(lo_b, device="cuda", requires_grad=True)
    thi = torch.tensor(hi_b, device="cuda", requires_grad=True)
    trat = torch.tensor(case.rating, device="cuda", requires_grad=True)
    obj_lo, obj_hi = ibp_bound(gpu, tlo, thi, trat)
    loss = (obj_hi * torch.tensor(w_hi, device="cuda")).sum() + \
        (obj_lo * torch.tensor(w_lo, device="cuda")).sum()
    loss.backward()
    # the oracle's hand gradients of both ends
    oh_lo, oh_hi, oh_r = O.grad_hi(case, sens, lo=lo_b, hi=hi_b)
    ol_lo, ol_hi, ol_r = O.grad_lo(case, sens, lo=lo_b, hi=hi_b)
    e_lo = w_hi[:, None] * oh_lo + w_lo[:, None] * ol_lo
    e_hi = w_hi[:, None] * oh_hi + w_lo[:, None] * ol_hi
    e_r = (w_hi[:, None] * oh_r + w_lo[:, None] * ol_r).sum(axis=0)
    sc = max(np.abs(e_lo).max(), np.abs(e_hi).max())
    np.testing.assert_allclose(tlo.grad.cpu().numpy(), e_lo, rtol=0, atol=1e-4 * sc)
    np.testing.assert_allclose(thi.grad.cpu().numpy(), e_hi, rtol=0, atol=1e-4 * sc)
    g_r = trat.grad.cpu().numpy()
    np.testing.assert_allclose(g_r, e_r, rtol=0, atol=1e-9 * max(1.0, np.abs(e_r).max()))
    # central differences of the oracle in the shared ratings, at lines whose
    # decisions sit far from their kinks in every box
    hr = 1e-3
    cb, rb = O.bus_box(case, lo_b, hi_b)
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    fb, fr = cb @ sens.phi.T, rb @ np.abs(sens.phi).T
    m = np.minimum.reduce([np.abs(np.abs(cent) - rad - case.rating).min(axis=1),
                           np.abs(np.abs(cent) + rad - case.rating).min(axis=1),
                           np.abs(np.abs(fb) - fr - case.rating), np.abs(np.abs(fb) + fr - case.rating)])
    ok = np.flatnonzero(m.min(axis=0) > 50 * hr)
    lines = np.union1d(ok[np.abs(e_r[ok]) > 0][:5], ok[:2])
    assert np.any(np.abs(e_r[lines]) > 0)
    base = O.bound(case, sens, lo=lo_b, hi=hi_b)
    # FP64 rounding of the two loss values, over the step
    noise = 1e-14 * (np.abs(w_hi * base.hi).sum() + np.abs(w_lo * base.lo).sum()) / (2 * hr)
    for l in lines:
        vals = []
        for sg in (1.0, -1.0):
            r = case.rating.copy()
            r[l] += sg * hr
            b = O.bound(dataclasses.replace(case, rating=r), sens, lo=lo_b, hi=hi_b)
            vals.append((w_hi * b.hi).sum() + (w_lo * b.lo).sum())
        fd = (vals[0] - vals[1]) / (2 * hr)
        assert abs(fd - g_r[l]) <= 1e-6 * max(1.0, abs(fd)) + noise, (l, fd, g_r[l], noise)
    gpu.close()
