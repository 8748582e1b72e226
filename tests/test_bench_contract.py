"""The JSON line of bench.py's reference arm (the oracle on the host cores), on
the 118-bus workload so that it runs in seconds: one line with the keys every
bench line carries, plus the reference arm's own (impl, cpu_baseline, e2e with
no copies).  Under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

COMMON = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
          "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def _run(extra_env=None):
    env = dict(os.environ, PYTHONPATH=ROOT, **(extra_env or {}))
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "1",
                           "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert COMMON <= set(d), COMMON - set(d)
    assert d["impl"] == "reference"
    assert d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    # a step is one bounded sample: ms_per_step is its wall time, value the
    # sample scaled to the whole bound (the sample is the whole bound at most)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert "sample" in d["step"]
    assert d["config"]["workload"].startswith("mesh118: 118 buses")
    # the same config object as the GPU arm prints for this workload
    sys.path.insert(0, ROOT)
    import bench
    from gen import make_config
    assert d["config"] == bench.bench_config(make_config(1), 1, 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "contingencies" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_ranks_print_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_stored_traffic_is_tied_to_the_kernel_sources():
    """A stored DRAM-traffic figure is reported only for the kernel sources it
    was measured on; after any change to them the bench reports null."""
    sys.path.insert(0, ROOT)
    import bench
    sha = bench.kernel_sources_sha()
    assert len(sha) == 16
    key = (3, 0, True, True)
    saved = dict(bench.MEASURED_TRAFFIC)
    try:
        bench.MEASURED_TRAFFIC[key] = (1.0e9, sha)
        assert bench.measured_traffic(key) == (1.0e9, f"ncu capture of kernel sources {sha}")
        bench.MEASURED_TRAFFIC[key] = (1.0e9, "0" * 16)
        value, note = bench.measured_traffic(key)
        assert value is None and note.startswith("stale")
        assert bench.measured_traffic((9, 9, False, False))[0] is None
    finally:
        bench.MEASURED_TRAFFIC.clear()
        bench.MEASURED_TRAFFIC.update(saved)
