"""Ragged networks (sizes from {73, 300, 500, 1000, 2000} buses, 16 sub-boxes
each): forward and backward through the autograd.Function, with the gradient
checked against FP64 central finite differences of the oracle on 8 sampled
networks (1e-4 relative, kink-free boxes and steps)."""
import numpy as np
import pytest

import oracle as O
from gen import make_ragged_batch

pytestmark = pytest.mark.gpu


def test_ragged_autograd_fd_on_8_networks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    from paper_2511_15624_gb300.autograd import ibp_bound
    from tests.test_gpu_adjoint import _kink_free
    nets = make_ragged_batch()  # the 64-network workload, 16 sub-boxes each
    small = [n for n in nets if n.n_bus <= 500]
    rng = np.random.default_rng(8)
    picked = [small[i] for i in rng.choice(len(small), 8, replace=False)]
    checked = 0
    for net in picked:
        sens = O.sensitivities(net)
        gpu = P.Case(net, device=0)
        # forward and backward of the 16-box workload through the autograd.Function
        lo = torch.tensor(net.box_lo, device="cuda", requires_grad=True)
        hi = torch.tensor(net.box_hi, device="cuda", requires_grad=True)
        _, obj_hi = ibp_bound(gpu, lo, hi)
        obj_hi.sum().backward()
        glo, ghi = lo.grad.cpu().numpy(), hi.grad.cpu().numpy()
        assert np.isfinite(glo).all() and np.isfinite(ghi).all()
        # FD check at a kink-free box: one of the 16, else a seeded sub-box
        cand = [(net.box_lo[j], net.box_hi[j], glo[j], ghi[j]) for j in range(net.n_box)]
        lo0, hi0 = net.box_lo.min(axis=0), net.box_hi.max(axis=0)
        for _ in range(40):
            a = lo0 + 0.45 * rng.random(net.n_dev) * (hi0 - lo0)
            b = hi0 - 0.45 * rng.random(net.n_dev) * (hi0 - lo0)
            cand.append((np.minimum(a, b), np.maximum(a, b), None, None))
        done = False
        for blo, bhi, g_lo, g_hi in cand:
            ok, h = _kink_free(net, sens, blo, bhi)
            if not ok:
                continue
            if g_lo is None:
                tl = torch.tensor(blo[None], device="cuda", requires_grad=True)
                th = torch.tensor(bhi[None], device="cuda", requires_grad=True)
                _, oh = ibp_bound(gpu, tl, th)
                oh.sum().backward()
                g_lo, g_hi = tl.grad.cpu().numpy()[0], th.grad.cpu().numpy()[0]
            ptr = np.concatenate([[0], np.cumsum(np.concatenate([net.gen_nseg, net.load_nseg]))])
            bk = np.concatenate([net.gen_bkpt, net.load_bkpt])
            ok_dims = [d for d in range(net.n_dev)
                       if np.min(np.abs(np.concatenate([bk[ptr[d]:ptr[d + 1]] - blo[d],
                                                        bk[ptr[d]:ptr[d + 1]] - bhi[d]]))) > 20 * h]
            if not ok_dims:
                continue
            dims = rng.choice(ok_dims, min(4, len(ok_dims)), replace=False)
            o_lo, o_hi, _ = O.grad_hi(net, sens, lo=blo[None], hi=bhi[None])
            scale = max(np.abs(o_lo).max(), np.abs(o_hi).max())
            for d in dims:
                for which, g in (("lo", g_lo), ("hi", g_hi)):
                    ap, bp, am, bm = blo.copy(), bhi.copy(), blo.copy(), bhi.copy()
                    if which == "lo":
                        ap[d] += h
                        am[d] -= h
                    else:
                        bp[d] += h
                        bm[d] -= h
                    fd = (O.bound(net, sens, lo=ap[None], hi=bp[None]).hi[0]
                          - O.bound(net, sens, lo=am[None], hi=bm[None]).hi[0]) / (2 * h)
                    assert abs(fd - g[d]) <= 1e-4 * max(abs(fd), 1e-3 * scale), (net.name, which, d)
            done = True
            break
        checked += done
    assert checked == 8
