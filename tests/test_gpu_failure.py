"""Allocation failure, forced on the host (no GPU fault): with the library's
allocation limit set, case creation and workspace growth return IBP_ENOMEM,
and the case stays usable once the limit is lifted -- the next call rebuilds
its workspace and gives the same bounds as before."""
import numpy as np
import pytest

from gen import make_config
from gen.cases import time_index_boxes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    yield pkg
    pkg._abi.ibp_set_alloc_limit(0)


def test_create_fails_cleanly(P):
    P._abi.ibp_set_alloc_limit(1 << 20)
    try:
        with pytest.raises(P.IBPError) as ei:
            P.Case(make_config(2), device=0)
        assert ei.value.status == P._abi.IBP_ENOMEM
    finally:
        P._abi.ibp_set_alloc_limit(0)
    P.Case(make_config(1), device=0).close()


def test_workspace_growth_fails_and_recovers(P):
    case = make_config(1)
    many = time_index_boxes(case, 64, seed=5)
    gpu = P.Case(case, device=0)
    lo1, hi1, err1 = gpu.bound(case.box_lo, case.box_hi)
    g1 = gpu.backward(case.box_lo, case.box_hi, np.ones(1))
    P._abi.ibp_set_alloc_limit(4096)
    try:
        with pytest.raises(P.IBPError) as ei:
            gpu.bound(many.box_lo, many.box_hi)
        assert ei.value.status == P._abi.IBP_ENOMEM
        with pytest.raises(P.IBPError) as ei:
            gpu.backward(many.box_lo, many.box_hi, np.ones(64))
        assert ei.value.status == P._abi.IBP_ENOMEM
    finally:
        P._abi.ibp_set_alloc_limit(0)
    # the workspace is rebuilt: same bits as before the failures
    lo2, hi2, err2 = gpu.bound(case.box_lo, case.box_hi)
    assert np.array_equal(lo1, lo2) and np.array_equal(hi1, hi2) and np.array_equal(err1, err2)
    g2 = gpu.backward(case.box_lo, case.box_hi, np.ones(1))
    np.testing.assert_allclose(g2[0], g1[0], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(g2[1], g1[1], rtol=1e-12, atol=1e-9)
    # and the larger call now works, agreeing with one-box calls
    lo, hi, err = gpu.bound(many.box_lo, many.box_hi)
    for j in (0, 31, 63):
        a, b, e = gpu.bound(many.box_lo[j:j + 1], many.box_hi[j:j + 1])
        assert abs(hi[j] - b[0]) <= err[j, 0] + e[0, 0]
        assert abs(lo[j] - a[0]) <= err[j, 1] + e[0, 1]
