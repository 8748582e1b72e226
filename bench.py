"""Benchmark: milliseconds per certified N-1 objective bound on the 8316-bus
synthetic network (10500 lines, 5000 non-islanding contingencies, 1100
generators, 5000 flexible loads), one box per bound.

One step = one full pass of the hot path (box -> bus intervals, base flows,
contingency flow intervals with fused penalty maps and reductions, objective
assembly) through the C ABI.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun), every rank bounds its own boxes of the same workload on
its own GPU (weak scaling, no data-path collective); rank 0 reports the
aggregate bounds per second as milliseconds per bound.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms per certified N-1 objective bound, 8316-bus"
# FP32 FMA throughput a register-only loop reaches on a GB300 (8 independent
# FFMA chains per thread, 8 CTAs of 256 threads per SM, CUDA events): 37.2e12
# lane-FMAs/s, reported beside the nominal peak as a second reference
FMA_LOOP_TFLOPS = 74.4

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# contingency kernel, from a one-pass ncu capture on the same workload; keyed
# by (config, tile-shape variant, screen on, network reduction on) and stored
# with the SHA-256 prefix of the kernel sources it was taken on
# (KERNEL_SOURCES).  Other workloads or tile shapes report null; a kernel
# build whose sources no longer match reports null with a note.
MEASURED_TRAFFIC = {(3, 0, True, True): (0.90089e9, "3f5249af420c2010")}
KERNEL_SOURCES = ("kernel_ctg.cu", "ctg_epilogue.cuh", "refine.cuh", "common.cuh", "internal.h")


def kernel_sources_sha():
    """SHA-256 prefix (16 hex digits) of the contingency kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_15624_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key):
    """(bytes per launch or None, note)."""
    hit = MEASURED_TRAFFIC.get(key)
    if hit is None:
        return None, "no ncu capture of this workload and tile shape"
    value, sha = hit
    now = kernel_sources_sha()
    if sha != now:
        return None, (f"stale: the stored capture was taken on kernel sources {sha or 'unrecorded'}, "
                      f"this build is {now}")
    return value, f"ncu capture of kernel sources {sha}"


def workload(case, cfg, nb):
    return (f"{case.name}: {case.n_bus} buses, {case.n_line} lines, {case.n_ctg} N-1 "
            f"contingencies, {case.n_gen} gens, {case.n_load} flexible loads, seed {1000 + cfg}, "
            f"{nb} box per bound")


def bench_config(case, cfg, nb):
    """The config object both arms print (the same keys and values)."""
    return {"workload": workload(case, cfg, nb), "boxes": nb,
            "l2": "no flush: the inputs exceed the cache (the streamed FP32 PTDF rows, 345 MB, "
                  "exceed the 129 MB L2 of the GPU arm)"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--config", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--variant", type=int, default=0,
                   help="contingency-kernel tile shape (0 = library default)")
    p.add_argument("--no-screen", action="store_true",
                   help="run every line through the contingency kernel (no paper-mode line screen)")
    p.add_argument("--no-reduction", action="store_true",
                   help="stream every active bus and line (no exact network reduction)")
    p.add_argument("--no-refine", action="store_true",
                   help="FP32 bounds only (no FP64 refinement of the terms that can reach obj_hi)")
    p.add_argument("--boxes", type=int, default=32,
                   help="box count of the batched measurement on the same network (0 = skip)")
    p.add_argument("--study", default="", choices=["", "bisection", "ragged", "linear"],
                   help="bisection: batched vs per-box gradient-guided bisection on mesh2000; "
                        "ragged: 64 uneven networks x 16 sub-boxes in one persistent launch; "
                        "linear: the linear relaxation bound on mesh2000 (time per iteration, "
                        "certified bound against iterations)")
    p.add_argument("--rounds", type=int, default=20)
    p.add_argument("--linear-config", type=int, default=2,
                   help="workload of --study linear (default: the 2000-bus case)")
    p.add_argument("--adjoint", action="store_true",
                   help="also time the adjoint of the upper bound (1 box and the batch)")
    p.add_argument("--cpu-seconds", type=float, default=20.0,
                   help="target CPU time of the oracle sample")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smmax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smmax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _oracle_sens(case):
    """The oracle's PTDF/LODF build and its wall time (excluded from every
    oracle timing, like the GPU case build)."""
    import oracle as O
    t0 = time.time()
    sens = O.sensitivities(case)
    return sens, time.time() - t0


def _oracle_sample(case, target_s: float, sens_and_s=None):
    """Time the oracle (as it stands) on a bounded sample of the bound: all lines
    against a subset of contingencies, then scale to the full contingency list.
    Returns (ms per bound, description, threads)."""
    import numpy as np

    import oracle as O
    sens, sens_s = sens_and_s if sens_and_s is not None else _oracle_sens(case)
    cb, rb = O.bus_box(case, case.box_lo, case.box_hi)
    # the parts outside the contingency loop, timed in full
    t0 = time.time()
    O.imbalance_interval(case, sens.phi, cb, rb)
    O.base_terms(case, sens.phi, cb, rb)
    O.cost_interval(case, case.box_lo[0], case.box_hi[0])
    rest_s = time.time() - t0
    threads = int(os.environ.get("IBP_ORACLE_THREADS", "0")) or len(os.sched_getaffinity(0))
    n = max(threads, 16)
    while True:
        sub = case.__class__(**{**case.__dict__, "ctg_line": case.ctg_line[:n]})
        ss = O.Sensitivities(phi=sens.phi, lodf=np.ascontiguousarray(sens.lodf[:, :n]),
                             ptdf_kk=sens.ptdf_kk[:n])
        t0 = time.time()
        O.ctg_terms(sub, ss, cb, rb)
        dt = time.time() - t0
        if dt >= 0.6 * target_s or n >= case.n_ctg:
            break
        n = min(case.n_ctg, int(n * max(1.2, target_s / max(dt, 1e-3))))
    per_bound = dt * case.n_ctg / n + rest_s
    desc = (f"oracle on {n} of {case.n_ctg} contingencies x all {case.n_line} lines x all "
            f"{case.n_bus} buses ({dt:.1f} s), scaled by {case.n_ctg}/{n}, plus base flows, "
            f"imbalance and costs in full ({rest_s:.1f} s); PTDF/LODF build ({sens_s:.1f} s) "
            f"excluded like the GPU case build")
    return per_bound * 1e3, desc, threads


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from gen import make_config
    case = make_config(args.config)
    sens_and_s = _oracle_sens(case)
    times, walls = [], []
    desc = ""
    threads = 1
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        ms, desc, threads = _oracle_sample(case, target_s=max(2.0, 60.0 / (args.warmup + args.steps)),
                                           sens_and_s=sens_and_s)
        if i >= args.warmup:
            times.append(ms)
            walls.append((time.time() - t0) * 1e3)
    v = statistics.median(times)
    # a step is one bounded sample of the bound: ms_per_step is its wall time,
    # value the sample scaled to the whole bound
    line = {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.median(walls), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "step": "one bounded sample of the bound (cpu_baseline.sample); value scales it to the "
                    "whole bound, ms_per_step is the sample's wall time",
            "config": bench_config(case, args.config, 1),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gb300(args):
    import numpy as np
    import torch

    import paper_2511_15624_gb300 as P
    from gen import make_config
    from paper_2511_15624_gb300.shard import max_over_ranks

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_config(args.config)
    gpu = P.Case(case, device=local)
    if args.variant:
        gpu.set_variant(args.variant)
    if args.no_screen:
        gpu.set_screen(False)
    if args.no_reduction:
        gpu.set_reduction(False)
    if args.no_refine:
        gpu.set_refine(False)
    info = gpu.info()
    # columns the contingency kernel streams: bus classes under the reduction
    reduced = (not args.no_reduction) and (info.n_bridges > 0 or info.n_bus_classes < info.n_active)
    n_cols = info.n_bus_classes if reduced else info.n_active
    nb = 1
    lo = torch.tensor(case.box_lo, device=dev)
    hi = torch.tensor(case.box_hi, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (device pointers, inputs resident in HBM)
    for _ in range(args.warmup):
        gpu.bound(lo, hi)
    gpu.sync()

    # (1) device-timed throughput
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            out = gpu.bound(lo, hi)
        stop.record(stream)
        barrier()
    gpu.sync()
    clocks = clk.summary()
    dev_ms = start.elapsed_time(stop)
    obj = [t.cpu().numpy() for t in out]

    # (2) per-kernel durations of the same launches, recorded by the library
    # with CUDA events on the launching stream
    gpu.set_timing(True)
    ktimes = []
    for _ in range(args.steps):
        gpu.bound(lo, hi)
        ktimes.append(gpu.last_timing())
    gpu.set_timing(False)
    # lines kept by the paper-mode screen (the contingency kernel's line count)
    n_live = gpu.last_live()[0]
    n_live_screened = n_live >= 0
    n_live = case.n_line if n_live < 0 else n_live
    ctg_ms = statistics.mean(t["contingency"] for t in ktimes)
    tot_k = {k: statistics.mean(t[k] for t in ktimes) for k in ktimes[0]}

    # (3) end to end through the public API with host buffers
    hlo = np.ascontiguousarray(case.box_lo)
    hhi = np.ascontiguousarray(case.box_hi)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gpu.bound(hlo, hhi)
    e2e_s = time.perf_counter() - t0

    # (4) batched: args.boxes time-index boxes of the same network in one call
    batched = None
    if args.boxes > 1:
        from gen.cases import time_index_boxes
        bcase = time_index_boxes(case, args.boxes, seed=2000 + args.config)
        blo = torch.tensor(bcase.box_lo, device=dev)
        bhi = torch.tensor(bcase.box_hi, device=dev)
        for _ in range(2):
            gpu.bound(blo, bhi)
        gpu.sync()
        bsteps = max(2, args.steps // 5)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(bsteps):
            gpu.bound(blo, bhi)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        bms = b0.elapsed_time(b1) / bsteps
        gpu.set_timing(True)
        gpu.bound(blo, bhi)
        bk = gpu.last_timing()
        gpu.set_timing(False)
        b_live = gpu.last_live()[0]
        b_live = case.n_line if b_live < 0 else b_live
        bflop = P.algorithmic_flop(case.n_ctg, b_live, n_cols, args.boxes)
        batched = {"boxes": args.boxes, "ms_per_call": bms, "ms_per_bound": bms / args.boxes,
                   "lines_kept_by_screen": b_live,
                   "contingency_kernel_ms": bk["contingency"],
                   "achieved_tflops": bflop / (bk["contingency"] * 1e-3) / 1e12}

    # (5) the paper's own bound (two-part contingency intervals) on the same box
    gpu.bound_paper(lo, hi)
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        pout = gpu.bound_paper(lo, hi)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    paper = {"ms_per_bound": p0.elapsed_time(p1) / args.steps,
             "obj_hi": float(pout[1][0]), "obj_lo": float(pout[0][0])}

    # (6) adjoint of obj_hi (forward with active-pair recording + backward
    # kernels), one box and, when measured, the batch
    adjoint = None
    if args.adjoint:
        def time_bwd(blo, bhi, reps):
            g = torch.ones(blo.shape[0], dtype=torch.float64, device=dev)
            gpu.backward(blo, bhi, g)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                gpu.backward(blo, bhi, g)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1) / reps
        adjoint = {"ms_per_call_1_box": time_bwd(lo, hi, max(2, args.steps // 4))}
        if batched is not None:
            adjoint["ms_per_call_%d_boxes" % args.boxes] = time_bwd(blo, bhi, 2)

    # the slowest rank sets the job time (no other exchange: every rank owns its bounds)
    dev_ms, e2e_ms = max_over_ranks([dev_ms, e2e_s * 1e3], device=dev)
    if rank != 0:
        return
    bounds = args.steps * nb * ws
    value = dev_ms / bounds
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA lanes x 2 x max clock
    flop = P.algorithmic_flop(case.n_ctg, n_live, n_cols, nb)
    achieved = flop / (ctg_ms * 1e-3) / 1e12
    traffic, traffic_note = measured_traffic((args.config, args.variant, not args.no_screen, reduced))
    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(case, args.config, nb),
        "detail": {"n_active_buses": info.n_active, "lines_kept_by_screen": n_live,
                   "network_reduction": {"on": reduced, "bus_classes": info.n_bus_classes,
                                         "bridges": info.n_bridges},
                   "interval_flows_per_s": case.n_ctg * case.n_line * nb / (value * 1e-3),
                   "kernel_ms": tot_k},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": traffic, "traffic_source": traffic_note,
                     # DRAM rate of the contingency kernel: measured bytes per launch over
                     # its live duration
                     "traffic_gbs": None if traffic is None else traffic / (ctg_ms * 1e-3) / 1e9,
                     "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                     "fma_loop_peak": {"value": FMA_LOOP_TFLOPS, "unit": "TFLOP/s",
                                       "frac": achieved / FMA_LOOP_TFLOPS,
                                       "source": "register-only FFMA loop on GB300 (measured)"}},
        "clocks": clocks,
        "e2e": {"value": e2e_ms / bounds, "unit": "ms",
                "h2d_bytes_per_step": int(2 * case.box_lo.nbytes),
                "d2h_bytes_per_step": int(4 * 8 * nb)},  # obj_lo, obj_hi, obj_err[2]
        # per step: box->bus and its per-box totals (one launch when the
        # active columns fit one block), base flows, contingency, partial
        # sums, assembly; screen, compaction and row gather; class radii under
        # the reduction; the FP64 refinement of the queued pairs and its
        # application
        "gpu_launches": (5 + (1 if info.n_active_pad > 256 else 0) + (3 if n_live_screened else 0)
                         + (1 if reduced else 0) + (0 if args.no_refine else 2)) * args.steps,
        "batched": None if batched is None else {
            **batched, "frac": batched["achieved_tflops"] / fp32_peak,
            "interval_flows_per_s": case.n_ctg * case.n_line * batched["boxes"] / (batched["ms_per_call"] * 1e-3)},
        "paper_mode": paper,
        "adjoint": adjoint,
        "objective": {"lo": float(obj[0][0]), "hi": float(obj[1][0]),
                      "err_hi": float(obj[2][0][0]), "err_lo": float(obj[2][0][1])},
    }
    if not args.no_cpu_baseline and ws == 1:
        ms, desc, threads = _oracle_sample(case, args.cpu_seconds)
        line["cpu_baseline"] = {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)


def _at_time(hist, t):
    """The gap a run had reached by wall time t (inf before its first round)."""
    g = float("inf")
    for r in hist:
        if r["s"] <= t:
            g = r["gap"]
    return g


def run_bisection_study(args):
    """Gap (UB - LB)/|LB| against wall seconds on the 2000-bus case, for the
    batched driver (one call per round for all leaves) and the per-box driver
    (one call per leaf), with IBP leaves (256-leaf frontier) and with
    linear-relaxation leaves (16-leaf frontier, 1000 iterations per round,
    children continuing their parent's slopes).  A third linear curve keeps
    the root box alone and continues its iteration by 1000 per round."""
    import torch

    import paper_2511_15624_gb300 as P
    from gen import make_config
    from paper_2511_15624_gb300.bisect import Bisection

    case = make_config(2)
    gpu = P.Case(case, device=0)
    lin_kw = dict(bound="linear", max_leaves=16, linear_iters=1000, linear_root_iters=10000)
    modes = {"ibp_batched": dict(max_leaves=256, batched=True),
             "ibp_single": dict(max_leaves=256, batched=False),
             "linear_batched": dict(lin_kw, batched=True),
             "linear_single": dict(lin_kw, batched=False)}
    out = {"study": "bisection", "workload": workload(case, 2, 1) + " (root box)",
           "rounds": args.rounds, "modes": {k: {kk: vv for kk, vv in v.items()} for k, v in modes.items()},
           "ibp_root": {}}
    lo0, hi0, err0 = gpu.bound(case.box_lo, case.box_hi)
    out["ibp_root"] = {"ub": float(hi0[0]), "err": float(err0[0, 0])}
    limit = 120.0  # seconds per curve
    for name, kw in modes.items():
        # warm-up rounds, not reported: the first multi-box calls and the
        # framework's first sorts and gathers over several leaves happen here
        Bisection(gpu, case.box_lo, case.box_hi, **kw).run(2)
        b = Bisection(gpu, case.box_lo, case.box_hi, **kw)
        hist = []
        for _ in range(args.rounds):
            r = b.step()
            hist.append({"round": r.round, "s": round(r.seconds, 4), "ub": r.ub, "lb": r.lb, "gap": r.gap,
                         "leaves": r.n_leaves, "bound_s": round(r.bound_seconds, 4),
                         "driver_s": round(r.round_seconds - r.bound_seconds, 4)})
            if r.seconds > limit:
                break
        out[name] = hist
    # the root box alone, its linear bound continued round by round
    lo = torch.tensor(case.box_lo, device="cuda")
    hi = torch.tensor(case.box_hi, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist, lb = [], -float("inf")
    for rnd in range(args.rounds + 1):
        ub, _, xp = gpu.bound_linear(lo, hi, 10000 if rnd == 0 else 1000, warm=rnd > 0)
        _, ph, pe = gpu.bound(xp, xp)
        lb = max(lb, float(ph[0] - pe[0, 0]))
        u = float(ub[0]) if rnd == 0 else min(hist[-1]["ub"], float(ub[0]))
        torch.cuda.synchronize()
        hist.append({"round": rnd + 1, "s": round(time.perf_counter() - t0, 4), "ub": u, "lb": lb,
                     "gap": (u - lb) / abs(lb), "leaves": 1})
    out["linear_root_only"] = hist
    # batched against per-box at equal wall time: at every round end of the
    # per-box run, the gap the batched run had reached by then (the two
    # kernels' certified bounds of the same leaves differ by about 1e-7 of
    # |LB|, hence a margin of 1e-6 in the gap); and the time each run took to
    # reach the per-box run's final gap
    cmp = {}
    for kind in ("ibp", "linear"):
        bh, sh = out[kind + "_batched"], out[kind + "_single"]
        pts = [(r["s"], _at_time(bh, r["s"]), r["gap"]) for r in sh]
        target = sh[-1]["gap"] + 1e-6
        t_b = next((r["s"] for r in bh if r["gap"] <= target), None)
        t_s = next((r["s"] for r in sh if r["gap"] <= target), None)
        cmp[kind] = {"points": len(pts), "batched_at_or_below": sum(1 for _, gb, gs in pts if gb <= gs),
                     "batched_at_or_below_1e-6": sum(1 for _, gb, gs in pts if gb <= gs + 1e-6),
                     "seconds_to_single_final_gap": {"batched": t_b, "single": t_s},
                     "ub_fall": (bh[0]["ub"] - bh[-1]["ub"]) / abs(bh[0]["ub"]),
                     "ub_fall_from_ibp_root": (out["ibp_root"]["ub"] - bh[-1]["ub"]) / abs(bh[-1]["ub"]),
                     "final": {"batched": {k: bh[-1][k] for k in ("s", "ub", "lb", "gap", "leaves")},
                               "single": {k: sh[-1][k] for k in ("s", "ub", "lb", "gap", "leaves")}}}
    out["equal_time"] = cmp
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)


def run_linear_study(args):
    """The linear relaxation bound (default: the 2000-bus case; see
    ``--linear-config``): device time per iteration for 1, 4 and 16 boxes,
    then the certified bound of the root box after 10000 iterations and after
    each further ``--rounds`` chunk of 1000 (warm calls), with the certified
    value f at the averaged primal point (the lower end of the gap) through
    the paper-mode bound."""
    import torch

    import paper_2511_15624_gb300 as P
    from gen import make_config

    cfg = args.linear_config
    case = make_config(cfg)
    gpu = P.Case(case, device=0)
    lo = torch.tensor(case.box_lo, device="cuda")
    hi = torch.tensor(case.box_hi, device="cuda")
    gpu.bound_linear(lo, hi, n_iter=100)  # the step sizes, first graph capture
    torch.cuda.synchronize()
    per_iter = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for nb in (1, 4, 16):
        L, H = lo.repeat(nb, 1), hi.repeat(nb, 1)
        gpu.bound_linear(L, H, n_iter=100)
        torch.cuda.synchronize()
        e0.record()
        gpu.bound_linear(L, H, n_iter=500)
        e1.record()
        torch.cuda.synchronize()
        per_iter[nb] = e0.elapsed_time(e1) / 500
    traj = []
    t0 = time.perf_counter()
    it, best, lb = 0, float("inf"), -float("inf")
    for rnd in range(args.rounds + 1):
        n = 10000 if rnd == 0 else 1000
        ub, err, xp = gpu.bound_linear(lo, hi, n_iter=n, warm=rnd > 0)
        it += n
        _, ph, pe = gpu.bound_paper(xp, xp)
        best = min(best, float(ub[0]))
        fx = float(ph[0] - pe[0, 0])
        lb = max(lb, fx)
        torch.cuda.synchronize()
        traj.append({"iterations": it, "s": round(time.perf_counter() - t0, 4), "ub": best,
                     "ub_err": float(err[0]), "f_at_point": fx, "lb": lb, "gap": (best - lb) / abs(lb)})
    _, ihi, _ = gpu.bound(lo, hi)
    out = {"study": "linear", "workload": workload(case, cfg, 1), "ms_per_iteration": per_iter,
           "ibp_ub": float(ihi[0]), "trajectory": traj}
    print(json.dumps(out), flush=True)


def run_ragged_study(args):
    """64 networks of uneven size, 16 sub-boxes each: one persistent launch of
    the contingency kernel replayed from a CUDA graph, against one call per case."""
    import torch

    import paper_2511_15624_gb300 as P
    from gen import make_ragged_batch

    nets = make_ragged_batch()
    t0 = time.perf_counter()
    cases = [P.Case(n, device=0) for n in nets]
    build_s = time.perf_counter() - t0
    if args.variant:
        for c in cases:
            c.set_variant(args.variant)
    los = [torch.tensor(n.box_lo, device="cuda") for n in nets]
    his = [torch.tensor(n.box_hi, device="cuda") for n in nets]
    P.bound_multi(cases, los, his)  # plan and workspaces, outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        P.bound_multi(cases, los, his, stream=s.cuda_stream)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.bound_multi(cases, los, his, stream=s.cuda_stream)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / args.steps
    # one call per case (multi-box kernel each), same boxes
    for c, lo, hi in zip(cases, los, his):
        c.bound(lo, hi)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        for c, lo, hi in zip(cases, los, his):
            c.bound(lo, hi)
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / args.steps
    flows = sum(n.n_ctg * n.n_line * n.n_box for n in nets)
    # work the launch does: non-bridge lines x bus classes under the reduction
    flop = 0.0
    for n, c in zip(nets, cases):
        inf = c.info()
        red = inf.n_bridges > 0 or inf.n_bus_classes < inf.n_active
        lines = n.n_line - inf.n_bridges if red else n.n_line
        cols = inf.n_bus_classes if red else inf.n_active
        flop += P.algorithmic_flop(n.n_ctg, lines, cols, n.n_box)
    sizes = {}
    for n in nets:
        sizes[n.n_bus] = sizes.get(n.n_bus, 0) + 1
    out = {"study": "ragged", "networks": len(nets), "boxes_per_network": nets[0].n_box,
           "bus_sizes": sizes, "case_build_s": build_s,
           "graph_ms_per_batch": graph_ms, "per_case_calls_ms_per_batch": seq_ms,
           "interval_flows_per_s": flows / (graph_ms * 1e-3),
           "algorithmic_tflops": flop / (graph_ms * 1e-3) / 1e12, "steps": args.steps}
    print(json.dumps(out), flush=True)


def main():
    args = _args()
    if args.study == "ragged":
        run_ragged_study(args)
        return
    if args.study == "bisection":
        run_bisection_study(args)
        return
    if args.study == "linear":
        run_linear_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
