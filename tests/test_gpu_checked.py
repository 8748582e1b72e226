"""The checked build (-DIBP_CHECK): every index guard in the contingency,
screen, gather and partial-sum kernels records an error instead of reading or
writing out of bounds.  A fresh process loads that build (IBP_LIB=check) and
runs each path of the library -- one box with and without the screen and the
network reduction, flows, many boxes, the paper-mode bound, the adjoint, many
networks in one launch, and the entry point without allocation -- on small
networks with ragged tiles; no guard may fire, and the results must agree
with the oracle."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import numpy as np, torch
    import oracle as O
    import paper_2511_15624_gb300 as P
    from gen import make_config, make_ragged_batch, make_network_case
    from gen.cases import time_index_boxes, make_two_core_case
    from tests.test_gpu_parity import check_objective
    assert P._abi.LIB_PATH.endswith("libibp_gb300_check.so")
    for case in (make_config(1), make_two_core_case(),
                 make_network_case("odd", 37, 61, 9, 20, seed=77)):
        sens = O.sensitivities(case)
        ref = O.bound(case, sens)
        rs = np.abs(ref.terms["costs"]).sum(axis=1)
        gpu = P.Case(case, device=0)
        for screen, reduce in ((True, True), (False, True), (True, False), (False, False)):
            gpu.set_screen(screen); gpu.set_reduction(reduce)
            lo, hi, err = gpu.bound(case.box_lo, case.box_hi)      # host mode reads the error word
            check_objective(lo, hi, err, ref, rel_scale=rs)
        gpu.set_screen(True); gpu.set_reduction(True)
        gpu.bound(case.box_lo, case.box_hi, flows=True)
        many = time_index_boxes(case, 20, seed=3)
        lo, hi, err = gpu.bound(many.box_lo, many.box_hi)
        check_objective(lo, hi, err, O.bound(many, sens), rel_scale=None if case.n_bus > 100 else
                        np.abs(O.bound(many, sens).terms["costs"]).sum(axis=1))
        plo, phi, perr = gpu.bound_paper(case.box_lo, case.box_hi)
        gpu.backward(many.box_lo, many.box_hi, np.ones(20))
        t = torch.tensor(case.box_lo[0], device="cuda")
        u = torch.tensor(case.box_hi[0], device="cuda")
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        P._abi.ibp_bound_noalloc(gpu.handle, t, u, out[0:1], out[1:2], out[2:4],
                                 stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        gpu.sync()
    nets = make_ragged_batch(n_net=6, n_sub=4, seed=77, sizes=(73, 300, 500))
    cases = [P.Case(n, device=0) for n in nets]
    los = [torch.tensor(n.box_lo, device="cuda") for n in nets]
    his = [torch.tensor(n.box_hi, device="cuda") for n in nets]
    P.bound_multi(cases, los, his)
    torch.cuda.synchronize()
    for c in cases:
        c.sync()                       # raises on a fired guard (IBP_EUNSOUND)
    print("checked build: no guard fired")
''')


def test_checked_build_paths():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_15624_gb300.build import build
    build(check=True)
    env = dict(os.environ, IBP_LIB="check", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no guard fired" in r.stdout
