"""Multi-rank path of the benchmark on CPU: two gloo ranks shard pair ranges
with no overlap, agree on the max-over-ranks step time, and sum FP64 moments."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2205_09900_gb300.shard import max_over_ranks, pair_range, sum_over_ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranges = [pair_range(s, rank, world, 1000) for s in range(3)]
        t = max_over_ranks(10.0 + rank, dist)
        m = sum_over_ranks([1.0, 2.0 * (rank + 1)], dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, ranges)
        out[rank] = (gathered, t, m.tolist())
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_is_disjoint_and_complete():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    gathered, t0, m0 = res[0]
    _, t1, m1 = res[1]
    assert t0 == t1 == 11.0                     # max over ranks, seen by both
    assert m0 == m1 == [2.0, 6.0]               # summed moments, seen by both
    covered = sorted(p for rank_ranges in gathered for (first, cnt) in rank_ranges for p in range(first, first + cnt))
    assert covered == list(range(3 * world * 1000))   # every pair once, no overlap


def test_single_process_identities():
    assert pair_range(2, 0, 1, 50) == (100, 50)
    assert max_over_ranks(3.5) == 3.5
    assert sum_over_ranks([1.0, 2.0]).tolist() == [1.0, 2.0]
