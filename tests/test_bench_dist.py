"""Host logic of the multi-rank benchmark path, on CPU with gloo (2 ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.0, 15.0][rank]
    mx = bench.reduce_max(ms, world)
    val = bench.aggregate(1000.0, mx, world)
    q.put((rank, mx, val))
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
    assert [r[1] for r in res] == [15.0, 15.0]                 # the slowest rank's time
    assert all(abs(r[2] - 2 * 1000.0 / 0.015) < 1e-6 for r in res)   # both replicas' edges


def _part_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(5)
    cost = np.sort(rng.integers(0, 5000, size=3000))[::-1].astype(np.uint64)   # per-item cost estimates
    per_item = rng.integers(0, 100, size=3000).astype(np.int64)                 # each item's partial count
    mine = bench.part_count_host(cost, per_item, rank, world)
    t = bench.sum_over_ranks_(torch.tensor([mine], dtype=torch.int64), world)
    q.put((rank, mine, int(t.item()), int(per_item.sum())))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_count_sums_to_the_whole(world):
    # each rank counts its cost-balanced range of the work list (the split of
    # eh_count_range, through the host entry point eh_range_bounds); the one
    # all-reduce gives every rank the whole count
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_part_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
    total = res[0][3]
    assert all(r[2] == total for r in res)
    assert sum(r[1] for r in res) == total
    assert all(r[1] > 0 for r in res)                           # every rank got work


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(10.0, 1000.0, 1) == 10.0


def test_step_stats():
    import bench
    st = bench.step_stats([10.0, 9.0, 30.0, 11.0, 10.0, 9.5, 1.0])
    assert st["min"] == 1.0 and st["max"] == 30.0 and st["median"] == 10.0
    assert abs(st["trimmed_mean"] - (9.0 + 9.5 + 10.0 + 10.0 + 11.0) / 5) < 1e-12
    assert bench.step_stats([4.0, 6.0])["trimmed_mean"] == 5.0
    assert bench.step_stats([7.0])["trimmed_mean"] == 7.0
