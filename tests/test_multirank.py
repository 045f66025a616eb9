"""Host logic of multi-rank runs on CPU: two gloo ranks (one process each) shard
the batched patches with no communication, and the timing reductions give the
slowest rank's time and the whole job's throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1908_03634_gb300 import sharding as S
from paper_1908_03634_gb300 import workloads as W


def test_shard_patches_partition_and_balance():
    cells = [n ** 3 for n in (32, 48, 64, 96, 128) for _ in range(19)] + [40 ** 3]
    for world in (1, 2, 3, 4, 8):
        sh = S.shard_patches(cells, world)
        assert sorted(i for s in sh for i in s) == list(range(len(cells)))
        loads = [sum(cells[i] for i in s) for s in sh]
        # longest-first greedy: the spread is at most the largest patch
        assert max(loads) - min(loads) <= max(cells)
    assert S.shard_patches([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        S.shard_patches([1], 0)


def test_shard_of_batched_workload_is_deterministic():
    from paper_1908_03634_gb300.workloads import batched_sizes
    sizes = batched_sizes(96, seed=3)
    cells = [a * b * c for a, b, c in sizes]
    assert S.shard_patches(cells, 4) == S.shard_patches(list(cells), 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cells = [n ** 3 for n in (32, 48, 64, 96, 128) for _ in range(5)]
        mine = S.shard_patches(cells, world)[rank]
        # every rank computed the same partition without talking: check by gathering
        got = [None] * world
        dist.all_gather_object(got, mine)
        ms_local = 10.0 + 5.0 * rank  # the slowest rank defines the job's time
        units_local = float(sum(cells[i] for i in mine))
        thr, ms = S.job_throughput(units_local, ms_local)
        q.put((rank, got, ms, thr, S.max_over_ranks(rank), S.sum_over_ranks(1.0)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = [n ** 3 for n in (32, 48, 64, 96, 128) for _ in range(5)]
    for rank, got, ms, thr, mx, n in res:
        assert sorted(i for s in got for i in s) == list(range(len(cells)))
        assert got == S.shard_patches(cells, world)
        assert ms == 15.0 and mx == 1.0 and n == 2.0
        assert thr == pytest.approx(sum(cells) / 15e-3)


def test_single_process_reductions_are_identity():
    assert S.max_over_ranks(3.5) == 3.5
    thr, ms = S.job_throughput(100.0, 20.0)
    assert ms == 20.0 and thr == pytest.approx(5000.0)
