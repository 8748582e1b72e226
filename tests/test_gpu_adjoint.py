"""GPU adjoint of the certified upper bound against the oracle: its
hand-derived gradient and FP64 central finite differences (1e-4 relative),
sampled at boxes away from every kink of the upper bound."""
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


def _kink_margin(case, sens, lo, hi):
    """Smallest distance of any active-set decision of obj_hi from its kink, in
    MW, and the step that keeps every decision fixed."""
    cb, rb = O.bus_box(case, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    m = np.abs(np.abs(cent[0]) - rad[0] - case.rating[None, :])
    fb = (cb @ sens.phi.T)[0]
    fr = (rb @ np.abs(sens.phi).T)[0]
    mb = np.abs(np.abs(fb) - fr - case.rating)
    mi = abs(abs(cb.sum()) - rb.sum())
    dist = min(m.min(), mb.min(), mi)
    hmax = np.abs(sens.phi).max() * (1 + np.abs(sens.lodf).max())
    return dist, dist / (20 * max(hmax, 1.0))


def _kink_free(case, sens, lo, hi):
    """(ok, step): every active-set decision of obj_hi sits farther from its
    kink than 1e-5 of the flow scale (the GPU's outward rounding is ~1e-6 of
    it, so GPU and oracle agree on the active set), and the FD step keeps all
    of them fixed."""
    cb, rb = O.bus_box(case, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    scale = float((np.abs(cent) + rad).max())
    dist, h = _kink_margin(case, sens, lo, hi)
    return dist > 1e-5 * (1.0 + scale), h


def _sub_boxes(case, n, seed, shrink=0.45):
    rng = np.random.default_rng(seed)
    lo0, hi0 = case.box_lo[0], case.box_hi[0]
    a = lo0 + shrink * rng.random((n, case.n_dev)) * (hi0 - lo0)
    b = hi0 - shrink * rng.random((n, case.n_dev)) * (hi0 - lo0)
    return np.minimum(a, b), np.maximum(a, b)


@pytest.mark.parametrize("cfg", [0, 1])
def test_adjoint_matches_oracle_and_fd(P, cfg):
    case = make_config(cfg)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    lo_b, hi_b = _sub_boxes(case, 24, 7 + cfg)
    picked = []
    for j in range(lo_b.shape[0]):
        dist, h = _kink_margin(case, sens, lo_b[j], hi_b[j])
        if dist > 1e-3 * (1 + np.abs(case.rating).max()):
            picked.append((j, h))
        if len(picked) == 3:
            break
    assert picked, "no kink-free sub-box drawn"
    for j, h in picked:
        lo, hi = lo_b[j:j + 1], hi_b[j:j + 1]
        glo, ghi, grat = gpu.backward(lo, hi, np.ones(1), want_rating=True)
        o_lo, o_hi, o_rat = O.grad_hi(case, sens, lo=lo, hi=hi)
        scale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
        np.testing.assert_allclose(glo, o_lo, rtol=0, atol=1e-4 * scale)
        np.testing.assert_allclose(ghi, o_hi, rtol=0, atol=1e-4 * scale)
        if o_rat is not None:
            np.testing.assert_allclose(grat, o_rat, rtol=0, atol=1e-9 * max(1.0, np.abs(o_rat).max()))
        # central finite differences of the oracle's FP64 upper bound
        rng = np.random.default_rng(100 + j)
        # coordinates whose endpoints sit away from every cost breakpoint
        ptr = np.concatenate([[0], np.cumsum(np.concatenate([case.gen_nseg, case.load_nseg]))])
        bk = np.concatenate([case.gen_bkpt, case.load_bkpt])
        ok_dims = [d for d in range(case.n_dev)
                   if np.min(np.abs(np.concatenate([bk[ptr[d]:ptr[d + 1]] - lo[0, d],
                                                    bk[ptr[d]:ptr[d + 1]] - hi[0, d]]))) > 20 * h]
        dims = ok_dims if len(ok_dims) <= 6 else rng.choice(ok_dims, 6, replace=False)
        for d in dims:
            for which, g in (("lo", glo), ("hi", ghi)):
                ap, bp, am, bm = lo[0].copy(), hi[0].copy(), lo[0].copy(), hi[0].copy()
                if which == "lo":
                    ap[d] += h
                    am[d] -= h
                else:
                    bp[d] += h
                    bm[d] -= h
                fp = O.bound(case, sens, lo=ap[None], hi=bp[None]).hi[0]
                fm = O.bound(case, sens, lo=am[None], hi=bm[None]).hi[0]
                fd = (fp - fm) / (2 * h)
                assert abs(fd - g[0, d]) <= 1e-4 * max(abs(fd), 1e-3 * scale), (which, d, fd, g[0, d])


def test_multi_box_adjoint_and_autograd(P):
    import torch
    from paper_2511_15624_gb300.autograd import ibp_bound
    case = make_config(1)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    lo_b, hi_b = _sub_boxes(case, 6, 21)
    w = np.linspace(0.5, 2.0, 6)
    glo, ghi = gpu.backward(lo_b, hi_b, w)
    for j in range(6):
        dist, _ = _kink_margin(case, sens, lo_b[j], hi_b[j])
        if dist <= 1e-3 * (1 + case.rating.max()):
            continue
        o_lo, o_hi, _ = O.grad_hi(case, sens, lo=lo_b[j:j + 1], hi=hi_b[j:j + 1])
        scale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
        np.testing.assert_allclose(glo[j], w[j] * o_lo[0], rtol=0, atol=1e-4 * w[j] * scale)
        np.testing.assert_allclose(ghi[j], w[j] * o_hi[0], rtol=0, atol=1e-4 * w[j] * scale)
    # the autograd.Function routes through the same adjoint
    tlo = torch.tensor(lo_b, device="cuda", requires_grad=True)
    thi = torch.tensor(hi_b, device="cuda", requires_grad=True)
    obj_lo, obj_hi = ibp_bound(gpu, tlo, thi)
    (obj_hi * torch.tensor(w, device="cuda")).sum().backward()
    # same adjoint; FP64 atomics may sum in another order (~1e-15 relative)
    gs = max(np.abs(glo).max(), np.abs(ghi).max())
    np.testing.assert_allclose(tlo.grad.cpu().numpy(), glo, rtol=0, atol=1e-9 * gs)
    np.testing.assert_allclose(thi.grad.cpu().numpy(), ghi, rtol=0, atol=1e-9 * gs)


def test_adjoint_on_the_2000_bus_case(P):
    """The adjoint of obj_hi at the 2000-bus root box against the oracle's hand
    gradient, device by device: within 1e-6 of the gradient's scale plus, per
    device, the contribution of the few active-set decisions that sit within
    1e-5 of the flow scale of their kink (each may be taken either way by the
    GPU's rounding; see the 64-network test's allowance); both the box
    endpoints and the rating gradient."""
    from tests.test_gpu_ragged import _fd_setup
    case = make_config(2)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    g_lo, g_hi, g_r = gpu.backward(case.box_lo, case.box_hi, np.ones(1), want_rating=True)
    o_lo, o_hi, o_r = O.grad_hi(case, sens)
    setup = _fd_setup(case, sens, case.box_lo[0], case.box_hi[0])
    assert setup is not None
    _, allow, n_near = setup
    gscale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
    dev = max(np.max(np.abs(g_lo[0] - o_lo[0]) - allow), np.max(np.abs(g_hi[0] - o_hi[0]) - allow))
    print(f"2000 buses: adjoint excess over the near-kink allowance {dev / gscale:.2e} of the scale "
          f"({n_near} decisions near a kink)")
    assert dev <= 1e-6 * gscale
    # rating gradient: z_f times the active counts; a near-kink decision moves one count
    rb, rc = O.grad_hi_ratings(case, sens, case.box_lo, case.box_hi)
    o_r = (rb + rc)[0]
    assert np.all(np.abs(g_r[0] - o_r) <= case.zeta_f * n_near + 1e-9 * case.zeta_f)
    gpu.close()
