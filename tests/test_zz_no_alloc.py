"""ibp_bound_noalloc: the one-box bound for callers that cannot allocate device
memory at bound time (stream capture, latency-bound host threads, programs
whose own allocator owns the device).  It must agree with ibp_bound on the
same case within the parity tolerance of the other GPU tests (1e-5 relative),
call after call, whether it runs first in a fresh process or after every other
test; it must contain the oracle's bound and lie within its own error bound of
it; a case too large for its fixed scratch array is refused before any device
work; a box with lo > hi poisons all four outputs with NaN.  The file name
sorts last so that a run stopping at the first failure has already run the
rest."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from gen import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    return P, torch


def _noalloc(P, torch, gpu, lo_row, hi_row, fill=float("nan")):
    lo = torch.tensor(lo_row, device="cuda")
    hi = torch.tensor(hi_row, device="cuda")
    out = torch.full((4,), fill, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P._abi.ibp_bound_noalloc(gpu.handle, lo, hi, out[0:1], out[1:2], out[2:4], stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("cfg", [1, 2])
def test_noalloc_matches_bound_on_two_calls(env, cfg):
    P, torch = env
    from tests.test_gpu_parity import check_objective
    case = make_config(cfg)
    gpu = P.Case(case, device=0)
    # the existing entry point with the tile shape whose round-up summation
    # layout (one add per bus, 32-bus chunks) matches this entry point's, so
    # that the a-priori error bounds are comparable too; this entry point has
    # no line screen or network reduction, so the reference call runs without
    # them as well
    gpu.set_variant(1)
    gpu.set_screen(False)
    gpu.set_reduction(False)
    ref_lo, ref_hi, ref_err = gpu.bound(case.box_lo, case.box_hi)
    oracle = O.bound(case, O.sensitivities(case))
    for call in range(2):
        o_lo, o_hi, e_hi, e_lo = _noalloc(P, torch, gpu, case.box_lo[0], case.box_hi[0])
        assert np.isfinite([o_lo, o_hi, e_hi, e_lo]).all(), (call, o_lo, o_hi, e_hi, e_lo)
        assert abs(o_hi - ref_hi[0]) <= 1e-5 * abs(ref_hi[0]), (call, o_hi, ref_hi[0])
        assert abs(o_lo - ref_lo[0]) <= 1e-5 * abs(ref_lo[0]), (call, o_lo, ref_lo[0])
        # the error bounds: obj_lo's (FP32 arithmetic, same summation layout)
        # within 1e-5 of each other; obj_hi's are FP64-sized after the
        # refinement in both, and agree within 1e-5 of the objective
        assert abs(e_hi - ref_err[0, 0]) <= 1e-5 * max(abs(ref_err[0, 0]), 1e-6 * abs(ref_hi[0])), \
            (call, e_hi, ref_err[0])
        assert abs(e_lo - ref_err[0, 1]) <= 1e-5 * abs(ref_err[0, 1]), (call, e_lo, ref_err[0])
        # against the oracle: sound, within 1e-5 and within its own error bound
        check_objective(np.array([o_lo]), np.array([o_hi]), np.array([[e_hi, e_lo]]), oracle)
    gpu.close()


def test_noalloc_bad_box_writes_nan(env):
    P, torch = env
    case = make_config(1)
    gpu = P.Case(case, device=0)
    lo = case.box_lo[0].copy()
    lo[3] = case.box_hi[0, 3] + 1.0          # lo > hi in one entry
    out = _noalloc(P, torch, gpu, lo, case.box_hi[0], fill=0.0)
    assert np.isnan(out).all(), out
    # the next call with a good box is clean again (the error word restarts at 0)
    out = _noalloc(P, torch, gpu, case.box_lo[0], case.box_hi[0])
    assert np.isfinite(out).all(), out
    gpu.close()


def test_noalloc_refuses_a_case_beyond_its_scratch(env):
    """The 5-bus ring with its 6 contingencies listed 349,867 times each
    (duplicates count twice, eq. (slack-sagg)) needs one partial-sum row block
    per tile of 128 lines x 64 contingencies: 32,801 tiles x 256 bytes, more
    than the 8 MiB array.  The call returns IBP_EINVAL and enqueues nothing, so
    the output keeps the value written before the call."""
    P, torch = env
    base = make_config(0)
    big = dataclasses.replace(base, ctg_line=np.tile(base.ctg_line, 349_867).astype(np.int32))
    assert -(-big.n_ctg // 64) * 256 > 8 << 20
    gpu = P.Case(big, device=0)
    lo = torch.tensor(big.box_lo[0], device="cuda")
    hi = torch.tensor(big.box_hi[0], device="cuda")
    out = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(P.IBPError) as ei:
        P._abi.ibp_bound_noalloc(gpu.handle, lo, hi, out[0:1], out[1:2], out[2:4],
                                 stream=torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == P._abi.IBP_EINVAL
    assert "scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 7.0)
    gpu.close()
