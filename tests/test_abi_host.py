"""Host-only checks of the C ABI: the library loads, exports every symbol that
include/ibp.h declares, and rejects bad inputs with a status code before any
device work (dry-run cases, device = -1)."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

from gen import find_bridges, make_config, make_network_case

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2511_15624_gb300.build import build
    build()
    import paper_2511_15624_gb300 as P
    return P


def test_exports_every_declared_symbol(pkg):
    hdr = open(os.path.join(ROOT, "include", "ibp.h")).read()
    names = set(re.findall(r"\b(ibp_[a-z_0-9]+)\s*\(", hdr))
    assert {"ibp_case_create", "ibp_bound", "ibp_bound_backward"} <= names
    lib = ctypes.CDLL(pkg._abi.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(pkg._abi.EXPORTED) == names


def _expect(P, status, fn):
    with pytest.raises(P.IBPError) as ei:
        fn()
    assert ei.value.status == status, str(ei.value)


def test_dry_run_validation(pkg):
    P = pkg
    c = make_config(1)
    P.dry_run_case(c)  # valid input passes
    bad = dataclasses.replace(c, line_from=c.line_from.copy())
    bad.line_from[3] = c.n_bus + 5
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, reactance=c.reactance.copy())
    bad.reactance[0] = -1.0
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, reactance=c.reactance.copy())
    bad.reactance[0] = np.nan
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, rating=c.rating.copy())
    bad.rating[2] = np.inf
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, ctg_line=np.array([0, c.n_line], np.int32))
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, gen_bkpt=c.gen_bkpt.copy(), gen_nseg=c.gen_nseg.copy())
    # two segments with non-increasing breakpoints on device 0
    bad = dataclasses.replace(c, gen_nseg=np.concatenate([[2], c.gen_nseg[1:]]).astype(np.int32),
                              gen_slope=np.concatenate([[1.0], c.gen_slope]),
                              gen_bkpt=np.concatenate([[5.0], c.gen_bkpt]))
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))
    bad = dataclasses.replace(c, line_to=c.line_to.copy())
    bad.line_to[0] = bad.line_from[0]
    _expect(P, P._abi.IBP_EINVAL, lambda: P.dry_run_case(bad))


def test_bridge_and_disconnected_rejected(pkg):
    P = pkg
    c = make_network_case("t", 12, 13, 3, 4, seed=5)
    br = find_bridges(c.n_bus, c.line_from, c.line_to)
    assert br.any()
    bad = dataclasses.replace(c, ctg_line=np.flatnonzero(br)[:1].astype(np.int32))
    _expect(P, P._abi.IBP_EISLAND, lambda: P.dry_run_case(bad))
    # drop a bridge line: the network falls apart
    keep = np.flatnonzero(~br | (np.arange(c.n_line) != np.flatnonzero(br)[0]))
    keep = np.array([l for l in range(c.n_line) if l != np.flatnonzero(br)[0]])
    disc = dataclasses.replace(c, line_from=c.line_from[keep], line_to=c.line_to[keep],
                               reactance=c.reactance[keep], rating=c.rating[keep],
                               ctg_line=np.zeros(0, np.int32))
    _expect(P, P._abi.IBP_EISLAND, lambda: P.dry_run_case(disc))


def test_box_validation_before_device(pkg):
    P = pkg
    c = make_config(0)
    d = P.dry_run_case(c)
    lo, hi = c.box_lo.copy(), c.box_hi.copy()
    lo[0, 1] = hi[0, 1] + 1.0
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound(lo, hi))
    lo = c.box_lo.copy()
    lo[0, 0] = np.nan
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound(lo, c.box_hi))
    _expect(P, P._abi.IBP_ENOTSUP, lambda: d.bound(c.box_lo, c.box_hi))
    with pytest.raises(ValueError):
        d.bound(c.box_lo[:, :3], c.box_hi[:, :3])
    # at most 65535 boxes per call (the box index is a grid's y dimension)
    many_lo = np.repeat(c.box_lo, 65536, axis=0)
    many_hi = np.repeat(c.box_hi, 65536, axis=0)
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound(many_lo, many_hi))
    _expect(P, P._abi.IBP_EINVAL, lambda: d.backward(many_lo, many_hi, np.ones(65536)))


def test_no_cpu_fallback_without_device(pkg):
    """On a machine without a GPU the product path fails loudly."""
    P = pkg
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _expect(P, P._abi.IBP_ECUDA, lambda: P.Case(make_config(0), device=0))


@pytest.mark.parametrize("which", ["cfg1", "cfg2", "sparse", "odd", "two-core"])
def test_network_reduction_partition(pkg, which):
    """The bus classes and bridge flags of the exact network reduction, checked
    against the oracle's FP64 PTDF and LODF (dry-run case, no GPU): bridges are
    the lines with PTDF_line[l,l] = 1 and have L[l,k] = 0 for every
    contingency; members of a class have equal PTDF columns on every non-bridge
    line, and the buses dropped with the slack's class have zero columns there."""
    import oracle as O
    P = pkg
    if which == "cfg1":
        c = make_config(1)
    elif which == "cfg2":
        c = make_config(2)
    elif which == "sparse":
        # few extra edges: many bridges and several small 2-edge-connected parts
        c = make_network_case("sparse", 160, 175, 30, 70, seed=91)
    elif which == "odd":
        c = make_network_case("odd", 37, 61, 9, 20, seed=77)
    else:
        # three meshed parts joined by bridges, slack at the end of a feeder
        from gen.cases import make_two_core_case
        c = make_two_core_case()
    case = P.dry_run_case(c)
    info = case.info()
    cls, br = case.reduction()
    phi = O.ptdf(c)
    fr, to = c.line_from, c.line_to
    diag = phi[np.arange(c.n_line), fr] - phi[np.arange(c.n_line), to]
    np.testing.assert_array_equal(br.astype(bool), np.abs(1.0 - diag) < 1e-9)
    assert info.n_bridges == int(br.sum())
    active = np.array(sorted((set(c.gen_bus.tolist()) | set(c.load_bus.tolist())) - {c.slack}))
    assert cls.shape == (active.size,) and info.n_active == active.size
    nb = ~br.astype(bool)
    scale = np.abs(phi).max()
    for j in range(info.n_bus_classes):
        cols = active[cls == j]
        assert cols.size >= 1
        d = np.abs(phi[nb][:, cols] - phi[nb][:, cols[:1]]).max()
        assert d <= 1e-12 * scale, (j, d)
    if np.any(cls < 0):
        assert np.abs(phi[nb][:, active[cls < 0]]).max() <= 1e-12 * scale
    assert set(np.unique(cls[cls >= 0]).tolist()) == set(range(info.n_bus_classes))
    if br.any() and c.n_ctg > 0:
        s = O.sensitivities(c)
        assert np.abs(s.lodf[br.astype(bool)]).max() <= 1e-9
    if which in ("sparse", "two-core"):
        assert info.n_bus_classes < info.n_active


def test_kernel_variant_lists(pkg):
    """The compiled kernel shapes (no GPU needed): one-box and multi-box ids are
    disjoint and unique, and each list holds the library's default for its box
    count (16 for one box, 29 for several)."""
    P = pkg
    one = P._abi.ibp_kernel_variants(False)
    many = P._abi.ibp_kernel_variants(True)
    assert len(set(one)) == len(one) and len(set(many)) == len(many)
    assert not set(one) & set(many)
    assert 16 in one and 29 in many


def test_linear_and_batched_adjoint_validation(pkg):
    """The linear-relaxation and batched-adjoint entry points check their
    arguments on the host, before any device work: boxes, iteration count,
    primal weight, warm-start index, adjoint side."""
    P = pkg
    c = make_config(0)
    d = P.dry_run_case(c)
    lo, hi = c.box_lo.copy(), c.box_hi.copy()
    bad = lo.copy()
    bad[0, 1] = hi[0, 1] + 1.0
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound_linear(bad, hi, n_iter=10))
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound_linear(lo, hi, n_iter=-1))
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound_linear(lo, hi, n_iter=10, primal_weight=0.0))
    _expect(P, P._abi.IBP_EINVAL, lambda: d.bound_linear(lo, hi, n_iter=10, primal_weight=float("nan")))
    ub, err, xp = np.empty(1), np.empty(1), np.empty_like(lo)
    _expect(P, P._abi.IBP_EINVAL, lambda: P._abi.ibp_bound_linear(d.handle, 1, lo, hi, 10, 0.01, ub, err, xp,
                                                                   ptr_mode=0, warm=-1))
    _expect(P, P._abi.IBP_ENOTSUP, lambda: d.bound_linear(lo, hi, n_iter=10))
    _expect(P, P._abi.IBP_ENOTSUP, lambda: d.linear_inherit(np.zeros(1, np.int32)))
    g = [np.ones(1)]
    out = [np.empty_like(lo)]
    _expect(P, P._abi.IBP_EINVAL, lambda: P._abi.ibp_bound_multi_backward(
        [d.handle], [1], [lo], [hi], g, out, out, side=2))
    _expect(P, P._abi.IBP_ENOTSUP, lambda: P._abi.ibp_bound_multi_backward(
        [d.handle], [1], [lo], [hi], g, out, out, side=0))
