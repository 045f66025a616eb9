"""Host logic of the multi-rank runs (one process per GPU).

A single projection solve does not shard here: ranks run independent solves
(replicas).  The batched workload -- independent patches of uneven sizes --
is split across ranks by cell count with no collective on the data path; the
only cross-rank operations are the timing reductions below (max of the timed
region over ranks, sum of the work done), taken after the work.
"""
from __future__ import annotations


def shard_patches(cells, world):
    """Assign patches to ranks, balancing the cell count: longest first, each
    to the rank with the fewest cells so far (ties: lowest rank; equal sizes:
    lowest patch index first), so every rank computes the same assignment
    without communicating.  Returns one sorted list of patch indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += int(cells[i])
    return [sorted(s) for s in out]


def _reduce(value, op):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value):
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX if dist.is_available() else None)


def sum_over_ranks(value):
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM if dist.is_available() else None)


def job_throughput(units_local, ms_local):
    """Whole-job throughput: the units all ranks processed / the slowest rank's
    time (units per second), and that time in ms."""
    ms = max_over_ranks(ms_local)
    units = sum_over_ranks(units_local)
    return units / (ms / 1e3), ms
