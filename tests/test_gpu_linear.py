"""ibp_bound_linear: the linear (CROWN-style) relaxation bound with slopes
optimised on the GPU.

* certified: at the slopes the GPU ends with (read back through
  ibp_case_linear_slopes), the oracle's own evaluation of the dual function
  (oracle.linear_bound, pinned by weak and strong LP duality) lies at or below
  the GPU's value, within the GPU's error bound plus the FP64 build allowance;
  it is also above the LP optimum (weak duality);
* it closes the gap: on the 118-bus box, 20000 iterations bring the bound
  within 2% of the LP optimum (IBP: 102% above it), and f at the averaged
  primal point within 2% below it."""
import numpy as np
import pytest

import oracle as O
from gen import make_config
from tests.test_gpu_parity import F64
from tests.test_oracle_ibp import _lp_optimum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as pkg
    pkg._abi.lib()
    return pkg


def _scale(case, lo, hi):
    """The size of the objective's terms (for the FP64 allowance)."""
    ref = O.bound(case, O.sensitivities(case), lo=lo[None], hi=hi[None])
    return float(np.abs(ref.terms["costs"]).sum() + case.zeta_inj * ref.terms["inj"][1][0]
                 + case.zeta_f * (ref.terms["fb"][1][0] + ref.terms["fc"][1][0]))


@pytest.mark.parametrize("cfg,n_iter", [(0, 3000), (1, 3000), (2, 1000)])
def test_linear_bound_is_certified(P, cfg, n_iter):
    case = make_config(cfg)
    sens = O.sensitivities(case)
    gpu = P.Case(case, device=0)
    ub, err, xp = gpu.bound_linear(case.box_lo, case.box_hi, n_iter=n_iter)
    a_c, a_b, a0 = gpu.linear_slopes(1)
    assert np.all(np.abs(a_c) <= 1) and np.all(np.abs(a_b) <= 1) and abs(a0[0]) <= 1
    ref = O.linear_bound(case, sens, case.box_lo[0], case.box_hi[0], a_b[0], a_c[0], a0[0],
                         factored=cfg == 2)
    d = F64 * _scale(case, case.box_lo[0], case.box_hi[0])
    print(f"cfg {cfg}: GPU linear bound {ub[0]:.9g} (err {err[0]:.3g}), oracle at its slopes {ref:.9g}")
    assert ub[0] >= ref - d, (ub[0], ref, d)
    assert ub[0] - ref <= err[0] + d, (ub[0] - ref, err[0], d)
    if cfg < 2:
        opt, _ = _lp_optimum(case, sens)
        assert ub[0] >= opt - d
    # the primal point lies in the box
    assert np.all(xp >= case.box_lo - 1e-9) and np.all(xp <= case.box_hi + 1e-9)
    gpu.close()


def test_linear_bound_closes_the_gap(P):
    case = make_config(1)
    sens = O.sensitivities(case)
    opt, _ = _lp_optimum(case, sens)
    gpu = P.Case(case, device=0)
    _, ibp_hi, _ = gpu.bound(case.box_lo, case.box_hi)
    ub, err, xp = gpu.bound_linear(case.box_lo, case.box_hi, n_iter=20000)
    lb = O.objective_point(case, sens, xp[0])
    # the certified value of f at the point, from the GPU (obj_hi - err_hi of the zero-width box)
    plo, phi, perr = gpu.bound(xp, xp)
    lb_gpu = phi[0] - perr[0, 0]
    print(f"LP optimum {opt:.7g}; IBP {ibp_hi[0]:.7g} ({(ibp_hi[0] - opt) / abs(opt):+.2%}); "
          f"linear {ub[0]:.7g} ({(ub[0] - opt) / abs(opt):+.2%}); f(x) {lb:.7g} "
          f"({(lb - opt) / abs(opt):+.2%}), certified {lb_gpu:.7g}")
    assert ub[0] >= opt - 1e-9 * abs(opt)
    assert ub[0] - opt <= 0.02 * abs(opt)
    assert opt - lb <= 0.02 * abs(opt)
    assert lb_gpu <= lb + 1e-9 * abs(lb) and lb - lb_gpu <= 1e-6 * abs(lb)
    gpu.close()
