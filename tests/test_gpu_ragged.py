"""The 64-network workload (sizes from {73, 300, 500, 1000, 2000} buses, all
non-bridge contingencies, 16 sub-boxes each) in one persistent launch
(ibp_bound_multi), and its batched adjoint (ibp_bound_multi_backward):

* forward: on one network of every size, all 16 boxes against the FP64 oracle
  at both ends -- sound, within 1e-5 of the oracle and within the reported
  error bound (plus the FP64 build allowance of the other parity tests);
* backward: for every network of the launch, the batched adjoint equals the
  per-case adjoint (ibp_bound_backward / ibp_bound_backward_lo on the same
  boxes: the same active pairs, summed in another order), at both ends;
  through the autograd.Function, the gradients of 8 networks sampled over all
  sizes match FP64 central finite differences of the oracle (1e-4 relative,
  with an allowance for the few active-set decisions that sit within 1e-5 of
  the flow scale of their kink)."""
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
    nets = make_ragged_batch()
    cases = [P.Case(n, device=0) for n in nets]
    los = [torch.tensor(n.box_lo, device="cuda") for n in nets]
    his = [torch.tensor(n.box_hi, device="cuda") for n in nets]
    yield P, torch, nets, cases, los, his
    for c in cases:
        c.close()


def test_ragged_forward_matches_oracle_at_every_size(env):
    from tests.test_gpu_parity import check_objective
    P, torch, nets, cases, los, his = env
    outs = P.bound_multi(cases, los, his)
    torch.cuda.synchronize()
    seen = {}
    for i, n in enumerate(nets):
        if n.n_bus in seen:
            continue
        seen[n.n_bus] = i
        lo, hi, err = (t.cpu().numpy() for t in outs[i])
        ref = O.bound(n, O.sensitivities(n))
        d_hi, d_lo = check_objective(lo, hi, err, ref)
        print(f"{n.name}: {n.n_box} boxes, hi dev {np.abs(d_hi).max():.2e}, lo dev {np.abs(d_lo).max():.2e}, "
              f"err_lo/|lo| {np.max(err[:, 1] / np.abs(ref.lo)):.2e}")
    assert sorted(seen) == [73, 300, 500, 1000, 2000]


@pytest.mark.parametrize("side", ["hi", "lo"])
def test_batched_backward_equals_per_case(env, side):
    """obj_hi's adjoint over all 64 networks; obj_lo's over the networks of at
    most 500 buses (its active set holds most pairs of a wide box, and its
    list is capped at 64M entries per case, fewer than 16 boxes of a 2000-bus
    network need)."""
    P, torch, nets, cases, los, his = env
    idx = list(range(len(nets))) if side == "hi" else [i for i, n in enumerate(nets) if n.n_bus <= 500]
    rng = np.random.default_rng(3 if side == "hi" else 4)
    gobj = [torch.tensor(rng.uniform(0.5, 1.5, nets[i].n_box), device="cuda") for i in idx]
    outs = P.bound_multi_backward([cases[i] for i in idx], [los[i] for i in idx], [his[i] for i in idx], gobj,
                                  side=side, want_rating=True)
    torch.cuda.synchronize()
    worst, flips = 0.0, 0
    for q, i in enumerate(idx):
        n, c = nets[i], cases[i]
        glo, ghi, grat = (t.cpu().numpy() for t in outs[q])
        # the per-case adjoint on the many-case path's line set (no screen)
        c.set_screen(False)
        rlo, rhi, rrat = c.backward(n.box_lo, n.box_hi, gobj[q].cpu().numpy(), want_rating=True, side=side)
        c.set_screen(True)
        scale = max(np.abs(rlo).max(), np.abs(rhi).max(), 1e-300)
        # the same active pairs, their sums in another order
        dev = max(np.abs(glo - rlo).max(), np.abs(ghi - rhi).max()) / scale
        worst = max(worst, dev)
        assert dev <= (1e-9 if side == "hi" else 1e-5), (n.name, side, dev)
        # rating gradient: z_f g times the line's active count; a pair at its
        # kink within the FP32 rounding of the two tile shapes may count on
        # one side only
        unit = n.zeta_f * gobj[q].cpu().numpy()[:, None]
        d = np.abs(grat - rrat) / unit
        assert np.all(d <= 2.0 + 1e-9), (n.name, d.max())
        flips += int((d > 0.5).sum())
    print(f"side {side}: {len(idx)} networks, worst relative deviation from the per-case adjoint "
          f"{worst:.2e}, rating entries differing by a pair {flips}")
    assert flips <= 1e-3 * sum(nets[i].n_box * nets[i].n_line for i in idx)


def _fd_setup(case, sens, lo, hi):
    """FD step and per-device allowance at a box.  Every active-set decision of
    obj_hi farther than delta = 1e-5 of the flow scale from its kink is kept
    fixed by the step; the few nearer ones (a handful in these networks) may
    be taken either way by the GPU's rounding or crossed inside the step, and
    each moves d obj_hi / d x_d by at most z_f |H_k[l, bus(d)]|, which the
    allowance sums (twice).  None when the imbalance decision is that near."""
    cb, rb = O.bus_box(case, lo[None], hi[None])
    cent, rad = O.all_ctg_flows(case, sens, cb, rb)
    scale = float((np.abs(cent) + rad).max())
    delta = 1e-5 * (1.0 + scale)
    m = np.abs(np.abs(cent[0]) - rad[0] - case.rating[None, :])
    fb = (cb @ sens.phi.T)[0]
    fr = (rb @ np.abs(sens.phi).T)[0]
    mb = np.abs(np.abs(fb) - fr - case.rating)
    mi = abs(abs(cb.sum()) - rb.sum())
    if mi < delta:
        return None
    far = min(m[m >= delta].min(initial=np.inf), mb[mb >= delta].min(initial=np.inf), mi)
    hmax = np.abs(sens.phi).max() * (1 + np.abs(sens.lodf).max())
    h = far / (20 * max(hmax, 1.0))
    dev_bus = np.concatenate([case.gen_bus, case.load_bus])
    kk, ll = np.nonzero(m < delta)
    H = sens.phi[ll][:, dev_bus] + sens.lodf[ll, kk][:, None] * sens.phi[case.ctg_line[kk]][:, dev_bus]
    allow = np.abs(H).sum(axis=0) + np.abs(sens.phi[np.nonzero(mb < delta)[0]][:, dev_bus]).sum(axis=0)
    return h, 2.0 * case.zeta_f * allow, len(kk) + int((mb < delta).sum())


def test_ragged_autograd_fd_on_8_networks_of_all_sizes(env):
    """Forward and backward of the whole 64-network launch through the
    autograd.Function; the gradients of 8 networks, sampled so that every
    size appears, against FP64 central differences of the oracle at their
    first sub-box (1e-4 relative plus the near-kink allowance of _fd_setup,
    on devices whose allowance is below 1e-5 of their gradient)."""
    from paper_2511_15624_gb300.autograd import ibp_bound_multi
    P, torch, nets, cases, los, his = env
    tl = [lo.clone().requires_grad_(True) for lo in los]
    th = [hi.clone().requires_grad_(True) for hi in his]
    outs = ibp_bound_multi(cases, tl, th)
    sum(o[1].sum() for o in outs).backward()
    rng = np.random.default_rng(8)
    by_size = {}
    for i, n in enumerate(nets):
        by_size.setdefault(n.n_bus, []).append(i)
    picked = [int(rng.choice(v)) for v in by_size.values()]
    rest = [i for i in range(len(nets)) if i not in picked]
    picked += [int(i) for i in rng.choice(rest, 8 - len(picked), replace=False)]
    assert {nets[i].n_bus for i in picked} == {73, 300, 500, 1000, 2000}
    for i in picked:
        net = nets[i]
        sens = O.sensitivities(net)
        glo, ghi = tl[i].grad.cpu().numpy(), th[i].grad.cpu().numpy()
        assert np.isfinite(glo).all() and np.isfinite(ghi).all()
        j = 0
        blo, bhi = net.box_lo[j], net.box_hi[j]
        setup = _fd_setup(net, sens, blo, bhi)
        assert setup is not None, net.name
        h, allow, n_near = setup
        o_lo, o_hi, _ = O.grad_hi(net, sens, lo=blo[None], hi=bhi[None])
        gscale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
        gmag = np.maximum(np.maximum(np.abs(o_lo[0]), np.abs(o_hi[0])), 1e-3 * gscale)
        ptr = np.concatenate([[0], np.cumsum(np.concatenate([net.gen_nseg, net.load_nseg]))])
        bk = np.concatenate([net.gen_bkpt, net.load_bkpt])
        ok_dims = [d for d in range(net.n_dev)
                   if allow[d] < 1e-5 * gmag[d]
                   and np.min(np.abs(np.concatenate([bk[ptr[d]:ptr[d + 1]] - blo[d],
                                                    bk[ptr[d]:ptr[d + 1]] - bhi[d]]))) > 20 * h]
        assert ok_dims, net.name
        for d in rng.choice(ok_dims, min(4, len(ok_dims)), replace=False):
            for which, g in (("lo", glo[j]), ("hi", ghi[j])):
                ap, bp, am, bm = blo.copy(), bhi.copy(), blo.copy(), bhi.copy()
                if which == "lo":
                    ap[d] += h
                    am[d] -= h
                else:
                    bp[d] += h
                    bm[d] -= h
                fd = (O.bound(net, sens, lo=ap[None], hi=bp[None]).hi[0]
                      - O.bound(net, sens, lo=am[None], hi=bm[None]).hi[0]) / (2 * h)
                assert abs(fd - g[d]) <= 1e-4 * max(abs(fd), 1e-3 * gscale) + allow[d], \
                    (net.name, which, d, fd, g[d], allow[d])
        print(f"{net.name}: FD checked on {min(4, len(ok_dims))} devices ({n_near} decisions near a kink, "
              f"{len(ok_dims)} of {net.n_dev} devices eligible)")


def test_batched_backward_in_cuda_graph():
    """The batched adjoint's plan is built outside capture; captured in a CUDA
    graph, a replay gives the direct call's gradients (up to the order of the
    FP64 atomic sums, 1e-9) and picks up new boxes written into the same input
    tensors."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    nets = make_ragged_batch(n_net=6, n_sub=4, seed=77, sizes=(73, 300, 500))
    cases = [P.Case(n, device=0) for n in nets]
    los = [torch.tensor(n.box_lo, device="cuda") for n in nets]
    his = [torch.tensor(n.box_hi, device="cuda") for n in nets]
    gobj = [torch.ones(n.n_box, dtype=torch.float64, device="cuda") for n in nets]
    ref = P.bound_multi_backward(cases, los, his, gobj)  # plan and workspaces, outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        P.bound_multi_backward(cases, los, his, gobj, stream=s.cuda_stream)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        outs = P.bound_multi_backward(cases, los, his, gobj, stream=s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    def close(x, y):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-12 * max(np.abs(y).max(), 1.0))

    for (a, b, _), (c, d, _) in zip(outs, ref):
        close(a, c)
        close(b, d)
    # new boxes in the same tensors: the replay follows them
    his[0].copy_(his[0] - 0.1 * (his[0] - los[0]))
    g.replay()
    torch.cuda.synchronize()
    direct = P.bound_multi_backward(cases[:1], los[:1], his[:1], gobj[:1])
    torch.cuda.synchronize()
    close(outs[0][0], direct[0][0])
    close(outs[0][1], direct[0][1])
    for c in cases:
        c.sync()
        c.close()


def test_lo_list_overflow_poisons_the_gradients(env):
    """obj_lo's active set holds most pairs of a wide box; 16 boxes of a
    2000-bus network need more entries than the case's list holds.  The batched
    adjoint then writes NaN into the overflowed boxes' gradients (no partial
    gradient is returned silently), and the case's sync reports IBP_ENOMEM."""
    P, torch, nets, cases, los, his = env
    i = next(i for i, n in enumerate(nets) if n.n_bus == 2000)
    gobj = [torch.ones(nets[i].n_box, dtype=torch.float64, device="cuda")]
    (glo, ghi, _), = P.bound_multi_backward([cases[i]], [los[i]], [his[i]], gobj, side="lo")
    torch.cuda.synchronize()
    glo, ghi = glo.cpu().numpy(), ghi.cpu().numpy()
    bad = np.isnan(glo).all(axis=1) & np.isnan(ghi).all(axis=1)
    print(f"{nets[i].name}: {int(bad.sum())} of {nets[i].n_box} boxes overflowed obj_lo's list")
    assert bad.any()
    assert np.all(np.isfinite(glo[~bad])) and np.all(np.isfinite(ghi[~bad]))
    with pytest.raises(P.IBPError) as ei:
        cases[i].sync()
    assert ei.value.status == P._abi.IBP_ENOMEM
    # the next call on the case starts clean
    cases[i].bound(nets[i].box_lo[:1], nets[i].box_hi[:1])
