"""Rank logic of the multi-GPU path, on CPU: box and network partitions, and a
world-size-2 gloo run in which each rank bounds its own boxes (oracle as the
per-rank worker) and the gathered result equals the single-process result."""
import os
import socket

import numpy as np
import pytest

from paper_2511_15624_gb300.shard import box_shard, gather_boxes, max_over_ranks, network_shard


@pytest.mark.parametrize("n_box,world", [(0, 1), (1, 2), (7, 2), (32, 8), (5, 8), (256, 3)])
def test_box_shard_covers_once(n_box, world):
    spans = [box_shard(n_box, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n_box
    for (a0, b0), (a1, _) in zip(spans, spans[1:]):
        assert b0 == a1
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1


def test_box_shard_rejects():
    with pytest.raises(ValueError):
        box_shard(4, 2, 2)
    with pytest.raises(ValueError):
        box_shard(-1, 0, 1)


def test_network_shard_lpt():
    rng = np.random.default_rng(7)
    work = rng.choice([73, 300, 500, 1000, 2000], size=64).astype(float) ** 2
    for world in (1, 2, 3, 8):
        parts = network_shard(work, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [work[p].sum() for p in parts]
        # Graham's bound for longest-first list scheduling
        lower = max(work.sum() / world, work.max())
        assert max(loads) <= 4.0 / 3.0 * lower + 1e-9
    # ties go to the lower rank, so equal work is dealt round-robin
    assert network_shard([1.0] * 4, 2) == [[0, 2], [1, 3]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle as O
    from gen import make_config
    from gen.cases import time_index_boxes

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = time_index_boxes(make_config(1), 7, seed=11)
        a, b = box_shard(case.n_box, rank, world)
        sens = O.sensitivities(case)
        res = O.bound(case, sens, case.box_lo[a:b], case.box_hi[a:b], nthreads=1)
        local = np.stack([res.lo, res.hi], axis=1)
        full = gather_boxes(local, case.n_box)
        t = max_over_ranks([float(rank), -float(rank)])
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), full=full, t=np.array(t))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_bound_their_boxes(tmp_path):
    import torch.multiprocessing as mp

    import oracle as O
    from gen import make_config
    from gen.cases import time_index_boxes

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    case = time_index_boxes(make_config(1), 7, seed=11)
    ref = O.bound(case, O.sensitivities(case), nthreads=1)
    want = np.stack([ref.lo, ref.hi], axis=1)
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        # gathering only concatenates, so every rank holds exactly the same values
        np.testing.assert_array_equal(z["full"], want)
        np.testing.assert_array_equal(z["t"], [1.0, 0.0])


def test_single_process_identity():
    x = np.arange(6.0).reshape(3, 2)
    np.testing.assert_array_equal(gather_boxes(x, 3), x)
    assert max_over_ranks([2.5, -1.0]) == [2.5, -1.0]
