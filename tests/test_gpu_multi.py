"""Many networks of uneven size in one persistent launch (ibp_bound_multi):
agreement with per-case bounds, parity with the oracle, and capture/replay in
a CUDA graph."""
import numpy as np
import pytest

import oracle as O
from gen import make_ragged_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    nets = make_ragged_batch(n_net=6, n_sub=4, seed=77, sizes=(73, 300, 500))
    cases = [P.Case(n, device=0) for n in nets]
    los = [torch.tensor(n.box_lo, device="cuda") for n in nets]
    his = [torch.tensor(n.box_hi, device="cuda") for n in nets]
    return P, torch, nets, cases, los, his


def test_multi_matches_per_case_and_oracle(env):
    P, torch, nets, cases, los, his = env
    outs = P.bound_multi(cases, los, his)
    torch.cuda.synchronize()
    for i, (n, c) in enumerate(zip(nets, cases)):
        c.sync()
        # the many-case launch reduces the network but does not screen lines:
        # the per-case call without the screen has the same work items, so only
        # the FP64 reduction order differs
        c.set_screen(False)
        lo1, hi1, e1 = c.bound(n.box_lo, n.box_hi)
        c.set_screen(True)
        lo, hi, err = (t.cpu().numpy() for t in outs[i])
        np.testing.assert_allclose(hi, hi1, rtol=1e-12, atol=0)
        np.testing.assert_allclose(lo, lo1, rtol=1e-12, atol=0)
        # the screened per-case bound moves only the rounding of the sums
        lo2, hi2, e2 = c.bound(n.box_lo, n.box_hi)
        assert np.all(np.abs(hi2 - hi) <= e2[:, 0] + err[:, 0])
        assert np.all(np.abs(lo2 - lo) <= e2[:, 1] + err[:, 1])
        if i < 2:
            ref = O.bound(n, O.sensitivities(n))
            scale = np.abs(ref.terms["costs"]).sum(axis=1)
            assert np.all(hi >= ref.hi - 1e-9 * scale) and np.all(lo <= ref.lo + 1e-9 * scale)
            assert np.all(np.abs(hi - ref.hi) <= 1e-5 * np.abs(ref.hi) + 1e-9 * scale)


@pytest.mark.parametrize("variant", [26, 28])
def test_multi_other_bodies(env, variant):
    """The many-case launch runs the body of the first case's variant: 26
    writes 8 partial rows per work item, 28 and the default 4.  Every body
    gives the default's bound up to the FP64 summation order, inside the
    reported error."""
    P, torch, nets, cases, los, his = env
    ref = [tuple(t.cpu().numpy() for t in o) for o in P.bound_multi(cases, los, his)]
    cases[0].set_variant(variant)
    try:
        outs = P.bound_multi(cases, los, his)
        torch.cuda.synchronize()
        for (lo0, hi0, e0), o in zip(ref, outs):
            lo, hi, err = (t.cpu().numpy() for t in o)
            assert np.all(np.abs(hi - hi0) <= e0[:, 0] + err[:, 0])
            assert np.all(np.abs(lo - lo0) <= e0[:, 1] + err[:, 1])
    finally:
        cases[0].set_variant(0)
    for c in cases:
        c.sync()


def test_multi_without_reduction(env):
    """With the reduction off, the many-case launch streams every line and
    active bus; it agrees with the per-case plain call the same way."""
    P, torch, nets, cases, los, his = env
    for c in cases:
        c.set_reduction(False)
    try:
        outs = P.bound_multi(cases, los, his)
        torch.cuda.synchronize()
        for i, (n, c) in enumerate(zip(nets, cases)):
            c.set_screen(False)
            lo1, hi1, e1 = c.bound(n.box_lo, n.box_hi)
            c.set_screen(True)
            lo, hi, err = (t.cpu().numpy() for t in outs[i])
            np.testing.assert_allclose(hi, hi1, rtol=1e-12, atol=0)
            np.testing.assert_allclose(lo, lo1, rtol=1e-12, atol=0)
    finally:
        for c in cases:
            c.set_reduction(True)


def test_multi_in_cuda_graph(env):
    P, torch, nets, cases, los, his = env
    ref = P.bound_multi(cases, los, his)  # builds the plan outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        P.bound_multi(cases, los, his, stream=s.cuda_stream)  # warm on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        outs = P.bound_multi(cases, los, his, stream=s.cuda_stream)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for (a, b, _), (c, d, _) in zip(outs, ref):
        assert torch.equal(a, c) and torch.equal(b, d)
    # replay picks up new boxes written into the same input tensors
    his[0].copy_(his[0] - 0.1 * (his[0] - los[0]))
    g.replay()
    torch.cuda.synchronize()
    # (per-case call on the many-case launch's path: no screen)
    cases[0].set_screen(False)
    lo1, hi1, _ = cases[0].bound(nets[0].box_lo, his[0].cpu().numpy())
    cases[0].set_screen(True)
    np.testing.assert_allclose(outs[0][1].cpu().numpy(), hi1, rtol=1e-12)


def test_multi_edge_cases():
    """The many-case launch and its batched adjoint with the cases a batch can
    hold at its edges: a network without contingencies, duplicated
    contingencies, separate contingency ratings, an odd line count, one box,
    and 17 boxes (a second, nearly empty box tile).  Forward against the
    oracle at the objective bar; adjoint against the per-case adjoint."""
    import dataclasses

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    from gen import make_config, make_network_case, split_boxes
    from tests.test_gpu_parity import check_objective

    base = make_config(1)
    rng = np.random.default_rng(11)
    nets = [
        dataclasses.replace(base, ctg_line=np.zeros(0, np.int32)),               # no contingencies
        dataclasses.replace(make_config(0), ctg_line=np.concatenate(
            [make_config(0).ctg_line, make_config(0).ctg_line[:2]]).astype(np.int32)),  # duplicates
        dataclasses.replace(base, rating_ctg=base.rating * 1.3),                 # separate ratings
        make_network_case("odd", 37, 61, 9, 20, seed=77),                       # odd line count
    ]
    # box counts 1, 17, 4, 17
    counts = [1, 17, 4, 17]
    boxed = []
    for n, nb in zip(nets, counts):
        if nb == 1:
            boxed.append(n)
            continue
        levels = int(np.ceil(np.log2(nb)))
        lo, hi = split_boxes(n.box_lo[0], n.box_hi[0], levels, rng)
        boxed.append(n.with_boxes(lo[:nb], hi[:nb]))
    cases = [P.Case(n, device=0) for n in boxed]
    los = [torch.tensor(n.box_lo, device="cuda") for n in boxed]
    his = [torch.tensor(n.box_hi, device="cuda") for n in boxed]
    outs = P.bound_multi(cases, los, his)
    torch.cuda.synchronize()
    for n, c, o in zip(boxed, cases, outs):
        c.sync()
        lo, hi, err = (t.cpu().numpy() for t in o)
        ref = O.bound(n, O.sensitivities(n))
        check_objective(lo, hi, err, ref, rel_scale=np.abs(ref.terms["costs"]).sum(axis=1))
    gobj = [torch.ones(n.n_box, dtype=torch.float64, device="cuda") for n in boxed]
    grads = P.bound_multi_backward(cases, los, his, gobj)
    torch.cuda.synchronize()
    for n, c, (glo, ghi, _) in zip(boxed, cases, grads):
        c.sync()
        c.set_screen(False)
        rlo, rhi = c.backward(n.box_lo, n.box_hi, np.ones(n.n_box))
        c.set_screen(True)
        scale = max(np.abs(rlo).max(), np.abs(rhi).max(), 1e-300)
        assert np.abs(glo.cpu().numpy() - rlo).max() <= 1e-9 * scale, n.name
        assert np.abs(ghi.cpu().numpy() - rhi).max() <= 1e-9 * scale, n.name
    for c in cases:
        c.close()


def test_linear_bound_without_contingencies():
    """The linear relaxation on a network without contingencies (only base
    lines and the imbalance carry slopes): certified against the oracle's
    evaluation at the GPU's slopes and above the LP optimum."""
    import dataclasses

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    from gen import make_config
    from tests.test_gpu_parity import F64, side_scales
    from tests.test_oracle_ibp import _lp_optimum

    case = dataclasses.replace(make_config(1), ctg_line=np.zeros(0, np.int32))
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    ub, err, xp = gpu.bound_linear(case.box_lo, case.box_hi, n_iter=5000)
    a_c, a_b, a0 = gpu.linear_slopes(1)
    ref = O.linear_bound(case, sens, case.box_lo[0], case.box_hi[0], a_b[0], a_c[0], a0[0])
    d = F64 * float(side_scales(O.bound(case, sens))[0][0])
    assert ub[0] >= ref - d and ub[0] - ref <= err[0] + d, (ub[0], ref)
    opt, _ = _lp_optimum(case, sens)
    assert ub[0] >= opt - d
    print(f"no contingencies: linear {ub[0]:.7g}, LP optimum {opt:.7g}")
    gpu.close()
