"""GPU vs oracle parity of the certified bound (calls go through the C ABI).

Tolerances (derived from the outward-rounding error analysis of the kernels):
* FP64 allowance: the library builds its own FP64 sensitivities (Cholesky on
  the GPU), the oracle its own (LU on the host).  Two independent FP64 builds
  moved obj_hi by at most 1.8e-13 of its hi-side terms and obj_lo by 1.3e-14
  of its lo-side terms on the 2000-bus workload (LU against Cholesky, both on
  the host; ``tests/test_oracle_fp64_builds.py`` keeps that measurement).  The
  tests allow F64 = 1e-10 of each side's own terms: for obj_hi the terms obj_hi
  is made of (|C_hi| + |G_lo| + z_inj s_inj,lo + z_f (s_fb,lo + s_fc,lo)), for
  obj_lo those of obj_lo;
* soundness: the GPU interval must contain the oracle's up to that allowance;
* objective: |gpu - oracle| <= 1e-5 |oracle| at both ends, and <= obj_err
  (the GPU's own error bound), each plus the same FP64 allowance;
* flows: each checked pair's interval [lo, hi] is compared at both ends with
  1e-5 of its magnitude max(|lo|, |hi|) where the FP32 operands do not cancel
  (s_kl <= 8 max(|lo|, |hi|)), else with 1e-5 s_kl, where
  s_kl = S_l + |L_lk| S_k with S_x = sum_b |Phi[x,b]| (|c_b| + r_b) is the
  magnitude of the FP32 operands combined for the pair (a centre or a
  post-outage flow that cancels to ~0 keeps an FP32-sized error relative to
  these operands), plus an absolute floor of 1e-12 max s_kl for lines whose
  exact flow is identically zero (both FP64 builds leave noise of that size
  there).
"""
import numpy as np
import pytest

import oracle as O
from gen import make_config, make_network_case, split_boxes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    return pkg


_SENS = {}


def _sens(key, case):
    if key not in _SENS:
        _SENS[key] = O.sensitivities(case)
    return _SENS[key]


F64 = 1e-10   # FP64 build allowance, relative to each side's own terms


def side_scales(ref):
    """The terms each end of the objective is made of, in absolute value:
    obj_hi = C_hi - G_lo - z_inj s_inj,lo - z_f (s_fb,lo + s_fc,lo) and
    obj_lo = C_lo - G_hi - z_inj s_inj,hi - z_f (s_fb,hi + s_fc,hi)."""
    C = np.atleast_2d(ref.terms["costs"])
    zi, zf = ref.terms["zeta"]
    hi_s = (np.abs(C[:, 1]) + np.abs(C[:, 2]) + zi * ref.terms["inj"][0]
            + zf * (ref.terms["fb"][0] + ref.terms["fc"][0]))
    lo_s = (np.abs(C[:, 0]) + np.abs(C[:, 3]) + zi * ref.terms["inj"][1]
            + zf * (ref.terms["fb"][1] + ref.terms["fc"][1]))
    return hi_s, lo_s


def check_objective(lo, hi, err, ref, rel=1e-5, rel_scale=None):
    """Soundness, 1e-5 agreement and error-bound coverage of both ends.

    rel_scale (default |oracle value|) is what the 1e-5 relative bar is taken
    of; the small synthetic networks whose objective cancels to about a tenth
    of its cost terms pass the cost scale instead.  Returns the measured
    relative deviations ((hi - ref.hi) / |ref.hi|, (lo - ref.lo) / |ref.lo|)."""
    hi_s, lo_s = side_scales(ref)
    d_hi, d_lo = F64 * hi_s, F64 * lo_s
    rs_hi = np.abs(ref.hi) if rel_scale is None else rel_scale
    rs_lo = np.abs(ref.lo) if rel_scale is None else np.maximum(rel_scale, np.abs(ref.lo))
    assert np.all(hi >= ref.hi - d_hi), ("unsound hi", hi, ref.hi, d_hi)
    assert np.all(lo <= ref.lo + d_lo), ("unsound lo", lo, ref.lo, d_lo)
    assert np.all(np.abs(hi - ref.hi) <= rel * rs_hi + d_hi), (hi, ref.hi)
    assert np.all(np.abs(lo - ref.lo) <= rel * rs_lo + d_lo), (lo, ref.lo)
    assert np.all(np.abs(hi - ref.hi) <= err[:, 0] + d_hi), (hi - ref.hi, err[:, 0])
    assert np.all(np.abs(lo - ref.lo) <= err[:, 1] + d_lo), (lo - ref.lo, err[:, 1])
    return (hi - ref.hi) / np.abs(ref.hi), (lo - ref.lo) / np.abs(ref.lo)


def bound_rows(ref, j):
    """Box j of an oracle Bound, as a one-box Bound."""
    terms = {}
    for k, v in ref.terms.items():
        if k == "zeta":
            terms[k] = v
        elif isinstance(v, tuple):
            terms[k] = tuple(t[j:j + 1] for t in v)
        else:
            terms[k] = v[j:j + 1]
    return O.Bound(lo=ref.lo[j:j + 1], hi=ref.hi[j:j + 1], terms=terms)


def flow_scale(case, sens, cb, rb, pk, pl):
    """Magnitude of the FP32 operands of pair (k, l): the centre and radius
    sums of both rows, sum_b |Phi| (|c_b| + r_b), combined through |L_lk|."""
    ab = np.abs(sens.phi)
    S = (np.abs(cb) + rb) @ ab.T
    kl = case.ctg_line[pk]
    L = np.abs(sens.lodf[pl, pk])
    return S[:, pl] + L[None, :] * S[:, kl]


def _worst(excess, pk, pl):
    i = np.unravel_index(np.argmax(excess), excess.shape)
    return f"worst excess {excess[i]:.3e} at box {i[0]} k={pk[i[1]]} l={pl[i[1]]}"


Q_CANCEL = 8.0  # s_kl / max(|lo|, |hi|) above which a pair counts as cancelling


def check_flows(case, sens, lo_box, hi_box, flo, fhi, pk, pl, rel=1e-5):
    """Flow intervals of the sampled pairs against the oracle (bars in the
    module docstring).  Returns (worst s_kl / max(|lo|, |hi|), share of pairs
    checked against the operand scale)."""
    cb, rb = O.bus_box(case, lo_box, hi_box)
    cent, rad = O.ctg_flows(case, sens, cb, rb, pk, pl)
    s = flow_scale(case, sens, cb, rb, pk, pl)
    # floor: both FP64 builds are accurate to ~1e-12 of the largest operand, so
    # lines whose exact flow is identically zero carry that much noise
    floor = 1e-12 * s.max()
    g_lo = flo[:, pk, pl]
    g_hi = fhi[:, pk, pl]
    mag = np.abs(cent) + rad
    ratio = s / np.maximum(mag, 1e-300)
    cancel = ratio > Q_CANCEL
    scale = np.where(cancel, s, mag)
    d = 1e-9 * s + floor
    assert np.all(g_lo <= cent - rad + d), _worst(g_lo - (cent - rad) - d, pk, pl)
    assert np.all(g_hi >= cent + rad - d), _worst((cent + rad) - g_hi - d, pk, pl)
    assert np.all(np.abs(g_lo - (cent - rad)) <= rel * scale + floor), \
        _worst(np.abs(g_lo - (cent - rad)) - rel * scale - floor, pk, pl)
    assert np.all(np.abs(g_hi - (cent + rad)) <= rel * scale + floor), \
        _worst(np.abs(g_hi - (cent + rad)) - rel * scale - floor, pk, pl)
    # the outaged line is exactly [0, 0]
    out = pl == case.ctg_line[pk]
    assert np.all(g_lo[:, out] == 0) and np.all(g_hi[:, out] == 0)
    live = ~np.broadcast_to(out, ratio.shape) & (mag > floor)
    worst = float(ratio[live].max()) if live.any() else 0.0
    share = float(cancel[live].mean()) if live.any() else 0.0
    print(f"flows: {pk.size} pairs x {ratio.shape[0]} boxes, worst s/max(|lo|,|hi|) = {worst:.3g}, "
          f"{100 * share:.2f}% checked against the operand scale")
    return worst, share


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_single_box_parity(P, cfg):
    case = make_config(cfg)
    sens = _sens(cfg, case)
    ref = O.bound(case, sens)
    gpu = P.Case(case, device=0)
    lo, hi, err, flo, fhi = gpu.bound(case.box_lo, case.box_hi, flows=True)
    check_objective(lo, hi, err, ref)
    if case.n_ctg * case.n_line <= 200_000:
        kk, ll = np.meshgrid(np.arange(case.n_ctg), np.arange(case.n_line), indexing="ij")
        pk, pl = kk.ravel(), ll.ravel()
    else:
        rng = np.random.default_rng(cfg)
        pk = rng.integers(0, case.n_ctg, 20000)
        pl = rng.integers(0, case.n_line, 20000)
        pl[:200] = case.ctg_line[pk[:200]]  # include outaged lines
    check_flows(case, sens, case.box_lo, case.box_hi, flo, fhi, pk, pl)


def test_device_pointer_mode_matches_host_mode(P):
    import torch
    case = make_config(1)
    gpu = P.Case(case, device=0)
    lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
    tlo = torch.tensor(case.box_lo, device="cuda")
    thi = torch.tensor(case.box_hi, device="cuda")
    dlo, dhi, derr = gpu.bound(tlo, thi)
    torch.cuda.synchronize()
    gpu.sync()
    assert np.array_equal(dlo.cpu().numpy(), lo) and np.array_equal(dhi.cpu().numpy(), hi)
    assert np.array_equal(derr.cpu().numpy(), err)
    # asking for flows turns the line screen off: same bound up to the rounding
    # order of the sums
    flo_, fhi_, ferr, fl, fh = gpu.bound(tlo, thi, flows=True)
    torch.cuda.synchronize()
    assert abs(float(fhi_[0]) - hi[0]) <= float(ferr[0, 0]) + err[0, 0]
    assert abs(float(flo_[0]) - lo[0]) <= float(ferr[0, 1]) + err[0, 1]
    # deterministic: a second call reproduces every bit
    lo2, hi2, err2 = gpu.bound(case.box_lo, case.box_hi)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)


def test_point_box_and_sub_boxes(P):
    case = make_config(1)
    sens = _sens(1, case)
    gpu = P.Case(case, device=0)
    rng = np.random.default_rng(3)
    x = case.box_lo[0] + rng.random(case.n_dev) * (case.box_hi[0] - case.box_lo[0])
    lo, hi, err = gpu.bound(x[None], x[None])
    f = O.objective_point(case, sens, x)
    assert lo[0] <= f + 1e-9 * abs(f) and f <= hi[0] + 1e-9 * abs(f)
    assert hi[0] - lo[0] <= 1e-5 * abs(f)
    # a few sub-boxes one by one
    slo, shi = split_boxes(case.box_lo[0], case.box_hi[0], 3, rng)
    ref = O.bound(case, sens, lo=slo, hi=shi)
    for j in range(slo.shape[0]):
        lo, hi, err = gpu.bound(slo[j:j + 1], shi[j:j + 1])
        check_objective(lo, hi, err, bound_rows(ref, j))


def test_edge_cases(P):
    # no contingencies at all
    case = make_config(1)
    import dataclasses
    nc = dataclasses.replace(case, ctg_line=np.zeros(0, np.int32))
    gpu = P.Case(nc, device=0)
    lo, hi, err = gpu.bound(nc.box_lo, nc.box_hi)
    ref = O.bound(nc, O.sensitivities(nc))
    check_objective(lo, hi, err, ref)
    # duplicated contingencies count twice, PWL costs with 3 segments, tiny network
    c0 = make_config(0, n_seg=3)
    dup = dataclasses.replace(c0, ctg_line=np.concatenate([c0.ctg_line, c0.ctg_line[:2]]).astype(np.int32))
    gpu = P.Case(dup, device=0)
    lo, hi, err = gpu.bound(dup.box_lo, dup.box_hi)
    check_objective(lo, hi, err, O.bound(dup, O.sensitivities(dup)))
    # separate contingency ratings
    rc = dataclasses.replace(case, rating_ctg=case.rating * 1.3)
    gpu = P.Case(rc, device=0)
    lo, hi, err = gpu.bound(rc.box_lo, rc.box_hi)
    check_objective(lo, hi, err, O.bound(rc, _sens(1, case)))
    # a network whose line count is not a multiple of anything, slack with devices
    odd = make_network_case("odd", 37, 61, 9, 20, seed=77)
    gpu = P.Case(odd, device=0)
    lo, hi, err = gpu.bound(odd.box_lo, odd.box_hi)
    check_objective(lo, hi, err, O.bound(odd, O.sensitivities(odd)))


def test_bad_box_on_device_reports_and_poisons(P):
    import torch
    case = make_config(0)
    gpu = P.Case(case, device=0)
    lo = case.box_lo.copy()
    lo[0, 2] = case.box_hi[0, 2] + 5.0
    dlo, dhi, derr = gpu.bound(torch.tensor(lo, device="cuda"), torch.tensor(case.box_hi, device="cuda"))
    torch.cuda.synchronize()
    with pytest.raises(P.IBPError) as ei:
        gpu.sync()
    assert ei.value.status == P._abi.IBP_EINVAL
    assert np.isnan(dhi.cpu().numpy()).all()
    # the case stays usable
    lo2, hi2, err2 = gpu.bound(case.box_lo, case.box_hi)
    assert np.isfinite(hi2).all()


def test_bounded_wait_times_out_cleanly(P):
    st = P._abi.ibp_selftest_wait_timeout(0, 1000)
    assert st == P._abi.IBP_ETIMEOUT
    # the context is still usable afterwards
    case = make_config(0)
    gpu = P.Case(case, device=0)
    lo, hi, err = gpu.bound(case.box_lo, case.box_hi)
    assert np.isfinite(hi).all()


@pytest.mark.parametrize("cfg", [1, 2])
def test_every_kernel_variant_parity(P, cfg):
    """Each compiled tile shape of the contingency kernel meets the same bar."""
    case = make_config(cfg)
    sens = _sens(cfg, case)
    ref = O.bound(case, sens)
    gpu = P.Case(case, device=0)
    rng = np.random.default_rng(10 + cfg)
    pk = rng.integers(0, case.n_ctg, 5000)
    pl = rng.integers(0, case.n_line, 5000)
    pl[:50] = case.ctg_line[pk[:50]]
    variants = P._abi.ibp_kernel_variants(False)
    assert len(variants) >= 2
    for vid in variants:
        gpu.set_variant(vid)
        lo, hi, err, flo, fhi = gpu.bound(case.box_lo, case.box_hi, flows=True)
        check_objective(lo, hi, err, ref)
        check_flows(case, sens, case.box_lo, case.box_hi, flo, fhi, pk, pl)


@pytest.mark.parametrize("cfg,n_sub", [(1, 5), (1, 16), (2, 20)])
def test_multi_box_parity(P, cfg, n_sub):
    """Many boxes in one call (ragged box tiles included) against the oracle,
    box by box, objective and flows."""
    case = make_config(cfg)
    sens = _sens(cfg, case)
    rng = np.random.default_rng(40 + n_sub)
    lo0, hi0 = case.box_lo[0], case.box_hi[0]
    a = lo0 + 0.5 * rng.random((n_sub, case.n_dev)) * (hi0 - lo0)
    b = hi0 - 0.5 * rng.random((n_sub, case.n_dev)) * (hi0 - lo0)
    lo_b, hi_b = np.minimum(a, b), np.maximum(a, b)
    lo_b[0] = hi_b[0]  # one point box
    ref = O.bound(case, sens, lo=lo_b, hi=hi_b)
    gpu = P.Case(case, device=0)
    for vid in P._abi.ibp_kernel_variants(True):
        gpu.set_variant(vid)
        lo, hi, err, flo, fhi = gpu.bound(lo_b, hi_b, flows=True)
        check_objective(lo, hi, err, ref)
        pk = rng.integers(0, case.n_ctg, 3000)
        pl = rng.integers(0, case.n_line, 3000)
        pl[:30] = case.ctg_line[pk[:30]]
        check_flows(case, sens, lo_b, hi_b, flo, fhi, pk, pl)
    # device pointers give the same bits as host pointers (same call shape:
    # no flows, so both run the line screen)
    import torch
    lo, hi, err = gpu.bound(lo_b, hi_b)
    dlo, dhi, derr = gpu.bound(torch.tensor(lo_b, device="cuda"), torch.tensor(hi_b, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(dhi.cpu().numpy(), hi) and np.array_equal(dlo.cpu().numpy(), lo)


def test_one_box_and_multi_box_agree(P):
    """The one-box and multi-box kernels bound the same box within tolerance."""
    case = make_config(2)
    gpu = P.Case(case, device=0)
    lo1, hi1, e1 = gpu.bound(case.box_lo, case.box_hi)
    two_lo = np.repeat(case.box_lo, 2, axis=0)
    two_hi = np.repeat(case.box_hi, 2, axis=0)
    lo2, hi2, e2 = gpu.bound(two_lo, two_hi)
    assert np.all(np.abs(hi2 - hi1[0]) <= 1e-5 * abs(hi1[0]))
    assert np.all(np.abs(lo2 - lo1[0]) <= 1e-5 * abs(lo1[0]))
    assert hi2[0] == hi2[1] and lo2[0] == lo2[1]
