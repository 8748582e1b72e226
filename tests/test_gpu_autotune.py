"""Tile-shape autotuner: times every shape, picks the fastest, caches it, and a
second case of the same shape reads the cache."""
import json
import os

import numpy as np
import pytest

from gen import make_config

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_caches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2511_15624_gb300 as P
    from paper_2511_15624_gb300.autotune import autotune
    case = make_config(1)
    path = os.path.join(tmp_path, "cache.json")
    for n_box in (1, 3):
        gpu = P.Case(case, device=0)
        lo = np.repeat(case.box_lo, n_box, axis=0)
        hi = np.repeat(case.box_hi, n_box, axis=0)
        r = autotune(gpu, lo, hi, cache_path=path, reps=2)
        assert not r["cached"]
        assert int(r["variant"]) in P._abi.ibp_kernel_variants(n_box > 1)
        assert r["ms"] == min(r["timed"].values())
        # the chosen shape still gives a bound
        a, b, e = gpu.bound(lo, hi)
        assert np.isfinite(b).all()
        gpu2 = P.Case(case, device=0)
        r2 = autotune(gpu2, lo, hi, cache_path=path)
        assert r2["cached"] and r2["variant"] == r["variant"]
    assert len(json.load(open(path))) == 2
