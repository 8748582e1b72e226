"""ibp_bound_noalloc: the one-box bound for callers that cannot allocate device
memory at bound time (stream capture, latency-bound host threads, programs
whose own allocator owns the device).  It must agree with ibp_bound on the
same case within the parity tolerance of the other GPU tests (1e-5 relative),
call after call, whether it runs first in a fresh process or after every other
test.  The file name sorts last so that a run stopping at the first failure has
already run the rest."""
import numpy as np
import pytest

from gen import make_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [1, 2])
def test_noalloc_matches_bound_on_two_calls(cfg):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P

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
    lo = torch.tensor(case.box_lo[0], device="cuda")
    hi = torch.tensor(case.box_hi[0], device="cuda")
    for call in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        P._abi.ibp_bound_noalloc(gpu.handle, lo, hi, out[0:1], out[1:2], out[2:4], stream=stream)
        torch.cuda.synchronize()
        o_lo, o_hi, e_hi, e_lo = out.cpu().numpy()
        assert np.isfinite([o_lo, o_hi, e_hi, e_lo]).all(), (call, o_lo, o_hi, e_hi, e_lo)
        assert abs(o_hi - ref_hi[0]) <= 1e-5 * abs(ref_hi[0]), (call, o_hi, ref_hi[0])
        assert abs(o_lo - ref_lo[0]) <= 1e-5 * abs(ref_lo[0]), (call, o_lo, ref_lo[0])
        assert abs(e_hi - ref_err[0, 0]) <= 1e-5 * abs(ref_err[0, 0]), (call, e_hi, ref_err[0])
        assert abs(e_lo - ref_err[0, 1]) <= 1e-5 * abs(ref_err[0, 1]), (call, e_lo, ref_err[0])
    gpu.close()
