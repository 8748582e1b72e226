"""Rank logic for running the bound on several GPUs, one process per GPU.

Every (contingency, line, box) interval is independent, and so are boxes and
networks.  The work therefore shards with no data-path exchange: each rank
bounds its own boxes (or its own networks) on its own GPU, and the ranks only
agree on timings and, when the caller wants every result everywhere, gather
the per-box FP64 results (a concatenation, no arithmetic, so the certified
values pass through unchanged).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def box_shard(n_box: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [start, stop) of the boxes owned by ``rank``; sizes differ by
    at most one and the first ``n_box % world`` ranks take the larger share."""
    if world < 1 or not 0 <= rank < world or n_box < 0:
        raise ValueError("need 0 <= rank < world and n_box >= 0")
    q, r = divmod(n_box, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def network_shard(work: Sequence[float], world: int) -> List[List[int]]:
    """Assign networks of uneven cost to ranks: longest first, each to the rank
    with the least work so far (ties to the lower rank).  Returns, per rank,
    the network indices in ascending order.  The largest rank load is at most
    4/3 of the optimum (Graham's bound for this rule)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(work, dtype=np.float64)
    if np.any(w < 0) or not np.all(np.isfinite(w)):
        raise ValueError("work must be finite and >= 0")
    load = np.zeros(world)
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(w)), key=lambda j: (-w[j], j)):
        r = int(np.argmin(load))
        out[r].append(i)
        load[r] += w[i]
    return [sorted(x) for x in out]


def _dist():
    import torch.distributed as dist

    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(values: Sequence[float], device=None) -> List[float]:
    """Element-wise maximum over all ranks (identity without a process group)."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    d = _dist()
    if d is not None:
        d.all_reduce(t, op=d.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def gather_boxes(local: np.ndarray, n_box: int) -> np.ndarray:
    """Concatenate per-rank results ``local`` [n_local, ...] (rank order, boxes
    as given by ``box_shard``) into the full [n_box, ...] array on every rank."""
    import torch

    d = _dist()
    local = np.ascontiguousarray(local, dtype=np.float64)
    if d is None:
        if local.shape[0] != n_box:
            raise ValueError("without a process group the local result must hold every box")
        return local.copy()
    world, rank = d.get_world_size(), d.get_rank()
    s0, s1 = box_shard(n_box, rank, world)
    if local.shape[0] != s1 - s0:
        raise ValueError(f"rank {rank} holds {local.shape[0]} boxes, expected {s1 - s0}")
    tail = local.shape[1:]
    width = -(-n_box // world)
    pad = np.zeros((width,) + tail)
    pad[: local.shape[0]] = local
    backend = d.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    src = torch.from_numpy(pad).to(dev)
    bufs = [torch.empty_like(src) for _ in range(world)]
    d.all_gather(bufs, src)
    parts = []
    for r in range(world):
        a, b = box_shard(n_box, r, world)
        parts.append(bufs[r][: b - a].cpu().numpy())
    return np.concatenate(parts, axis=0)


__all__ = ["box_shard", "network_shard", "max_over_ranks", "gather_boxes"]
