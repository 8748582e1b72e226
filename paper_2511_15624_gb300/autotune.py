"""Tile-shape autotuner for the contingency kernel, with a JSON cache.

For a case and a box count it times every compiled tile shape of the matching
kind (one-box or multi-box) with CUDA events on the call's stream, keeps the
fastest, and records it under a key made of the GPU name, the case sizes and
the box-count bucket.  Later cases of the same shape read the choice from the
cache without timing.
"""
from __future__ import annotations

import json
import os
from typing import Optional

import numpy as np

from . import _abi
from .case import Case

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                             "autotune_cache.json")


def _bucket(n_box: int) -> int:
    b = 1
    while b < n_box:
        b *= 2
    return b


def cache_key(case: Case, n_box: int, device_name: str) -> str:
    info = case.info()
    return (f"{device_name}|nl{info.n_line}|nc{info.n_ctg}|na{info.n_active}|"
            f"b{_bucket(n_box)}")


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def autotune(case: Case, box_lo, box_hi, cache_path: Optional[str] = None, reps: int = 3,
             force: bool = False) -> dict:
    """Pick the fastest tile shape for this case and box count; returns
    {"variant", "ms", "timed": {variant: ms}, "cached": bool}."""
    import torch
    path = cache_path or DEFAULT_CACHE
    lo = torch.as_tensor(np.atleast_2d(box_lo), dtype=torch.float64, device=f"cuda:{case.device}")
    hi = torch.as_tensor(np.atleast_2d(box_hi), dtype=torch.float64, device=f"cuda:{case.device}")
    n_box = int(lo.shape[0])
    name = torch.cuda.get_device_name(case.device)
    key = cache_key(case, n_box, name)
    cache = _load(path)
    if key in cache and not force:
        case.set_variant(int(cache[key]["variant"]))
        return {**cache[key], "cached": True}
    stream = torch.cuda.current_stream(case.device)
    timed = {}
    for vid in _abi.ibp_kernel_variants(n_box > 1):
        case.set_variant(vid)
        case.bound(lo, hi)  # warm-up (and first-use setup)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            case.bound(lo, hi)
        t1.record(stream)
        t1.synchronize()
        timed[vid] = t0.elapsed_time(t1) / reps
    best = min(timed, key=timed.get)
    case.set_variant(best)
    entry = {"variant": int(best), "ms": timed[best], "timed": {str(k): v for k, v in timed.items()}}
    cache = _load(path)
    cache[key] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return {**entry, "cached": False}


__all__ = ["autotune", "cache_key", "DEFAULT_CACHE"]
