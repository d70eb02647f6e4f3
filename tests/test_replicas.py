"""The N > 1 path of bench.py (replicas: one independent disk per rank, no
data-path collective), run as two gloo ranks on the CPU: the timing is the
slowest rank's, the aggregate counts every rank's moonlets, and the ranks'
disks differ (seed + rank)."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2310_20374_gb300 import diskgen
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = 10.0 + 5.0 * r                       # this rank's timed region
        t_max = bench.slowest_rank(dist, ms, w, device="cpu")
        d = diskgen.make_disk(1000, 2 + r)        # the bench's per-rank disk
        out[r] = (r, w, local, t_max, bench.replica_throughput(1000, 4, w, t_max * 1e-3), float(d["pos"][0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_slowest_and_count_all_replicas():
    world, port = 2, 29561
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rank, w, local, t_max, value, x0 = res[r]
        assert (rank, w, local) == (r, world, r)
        assert t_max == 15.0                      # the slower rank's 15 ms on both ranks
        assert value == pytest.approx(1000 * 4 * world / 0.015)
    assert res[0][5] != res[1][5]                 # different disks per rank


def test_single_rank_needs_no_collective():
    import bench
    assert bench.slowest_rank(None, 12.5, 1) == 12.5
    assert bench.replica_throughput(100000, 200, 1, 0.128) == pytest.approx(100000 * 200 / 0.128)
