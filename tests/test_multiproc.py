"""The N > 1 path without a GPU: two gloo ranks shard configurations the way
bench.py does (weak scaling, disjoint configuration ranges, no data-path
collective) and the summed counts equal one unsharded run; the timing
aggregate takes the slowest rank."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, k = bench.shard_range(rank, n)
    r = oracle.inspect(4, 16, p=0.25, seed=1, cfg0=b, n=k, mode="bfs", threads=1)
    su = oracle.site_updates(61, 16, r["verdict"], r["first_hit"], r["m_stop"])
    t = torch.tensor([float(r["verdict"].sum()), float(su)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    secs = torch.tensor([0.5 + rank], dtype=torch.float64)
    dist.all_reduce(secs, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((t.tolist(), float(secs.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_equals_single_run():
    world, n = 2, 300
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    (perc, su), tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = oracle.inspect(4, 16, p=0.25, seed=1, cfg0=0, n=world * n, mode="bfs")
    assert perc == float(whole["verdict"].sum())
    assert su == float(oracle.site_updates(61, 16, whole["verdict"], whole["first_hit"],
                                           whole["m_stop"]))
    assert tmax == 1.5
    assert bench.aggregate([10, 30], [1.0, 2.0]) == 20.0


def test_shard_ranges_are_disjoint_and_cover():
    n = 10_000
    ranges = [bench.shard_range(r, n) for r in range(8)]
    covered = np.concatenate([np.arange(b, b + k) for b, k in ranges])
    assert len(np.unique(covered)) == 8 * n and covered.min() == 0 and covered.max() == 8 * n - 1
