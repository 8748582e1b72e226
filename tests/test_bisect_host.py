"""The bisection driver's host logic on CPU tensors, with the oracle standing in
for the GPU case (its bound and its hand adjoint of obj_hi), on the 5-bus ring:
the leaves stay inside the root box and do not overlap, the upper bound never
rises and stays above f at every sampled point of the root box, the lower
bound never falls and never passes the upper bound, and a saved frontier
reloads to the same next round."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from gen import make_config
from paper_2511_15624_gb300.bisect import Bisection


class OracleCase:
    """bound() and backward() of the case API, computed by the oracle on one
    thread (its threaded sums add in scheduling order, so two calls on the same
    boxes could differ in the last bit, and the checkpoint test compares
    exactly)."""

    def __init__(self, case):
        self.case = case
        self.sens = O.sensitivities(case)
        self.device = 0

    def bound(self, lo, hi):
        r = O.bound(self.case, self.sens, lo.numpy(), hi.numpy(), nthreads=1)
        # the oracle's FP64 bound: no separate rounding allowance
        return torch.tensor(r.lo), torch.tensor(r.hi), torch.zeros(lo.shape[0], 2, dtype=torch.float64)

    def backward(self, lo, hi, g):
        gl, gh, _ = O.grad_hi(self.case, self.sens, lo.numpy(), hi.numpy(), nthreads=1)
        w = g.numpy()[:, None]
        return torch.tensor(gl * w), torch.tensor(gh * w)


@pytest.fixture(scope="module")
def ring():
    case = make_config(0)
    oc = OracleCase(case)
    yield case, oc
    # the oracle's thread count is process-wide: give the later tests all cores again
    O.bound(case, oc.sens, nthreads=len(os.sched_getaffinity(0)))


def _run(ring, batched, rounds):
    case, oc = ring
    b = Bisection(oc, case.box_lo, case.box_hi, max_leaves=16, batched=batched,
                  device=torch.device("cpu"), split_per_round=4)
    b.run(rounds)
    return b


def test_frontier_and_bounds(ring):
    case, oc = ring
    b = _run(ring, True, 6)
    ubs = [r.ub for r in b.history]
    lbs = [r.lb for r in b.history]
    assert all(u1 <= u0 for u0, u1 in zip(ubs, ubs[1:]))
    assert all(l1 >= l0 for l0, l1 in zip(lbs, lbs[1:]))
    assert all(l <= u for l, u in zip(lbs, ubs))
    lo, hi = b.lo.numpy(), b.hi.numpy()
    assert lo.shape[0] >= 2
    root_lo, root_hi = case.box_lo[0], case.box_hi[0]
    assert np.all(lo >= root_lo) and np.all(hi <= root_hi) and np.all(lo <= hi)
    # leaves overlap at most on a face
    for i in range(len(lo)):
        for j in range(i + 1, len(lo)):
            assert np.any(np.minimum(hi[i], hi[j]) <= np.maximum(lo[i], lo[j]))
    # UB bounds f over the whole root box
    rng = np.random.default_rng(5)
    for _ in range(200):
        x = root_lo + rng.random(root_lo.shape) * (root_hi - root_lo)
        assert O.objective_point(case, oc.sens, x) <= b.ub + 1e-9 * abs(b.ub)


def test_checkpoint_reloads_to_the_same_round(ring, tmp_path):
    case, oc = ring
    a = _run(ring, True, 3)
    path = str(tmp_path / "frontier.npz")
    a.save(path)
    b = Bisection.load(oc, path, max_leaves=16, batched=True, device=torch.device("cpu"),
                       split_per_round=4)
    assert b.round == a.round and b.ub == a.ub and b.lb == a.lb
    ra, rb = a.step(), b.step()
    assert (ra.ub, ra.lb, ra.n_leaves) == (rb.ub, rb.lb, rb.n_leaves)
    assert torch.equal(a.lo, b.lo) and torch.equal(a.hi, b.hi)


def test_single_mode_follows_the_same_rules(ring):
    """One call per box gives the same frontier as the batched calls, up to
    the summation order of the oracle's vectorised sums."""
    a = _run(ring, True, 4)
    b = _run(ring, False, 4)
    assert a.lo.shape == b.lo.shape
    np.testing.assert_allclose(a.ub, b.ub, rtol=1e-12)
    np.testing.assert_allclose(a.lb, b.lb, rtol=1e-12)
