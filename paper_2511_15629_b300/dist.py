"""Host-side logic of multi-GPU runs (one process per GPU).

The storage problems of a portfolio are independent (one value function per
asset), so a portfolio shards across ranks with no collective on the data
path: each rank solves its own assets.  A single asset does not shard (its
stages are sequential and every stage needs the neighbouring SoC rows), so a
single-asset job runs as independent replicas.  The only collectives are
the timing ones: a barrier around the timed region and the maximum of the
ranks' times (the job ends when the slowest rank ends).
"""
from __future__ import annotations

from typing import List, Sequence


def shard_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment of units (assets) to `world` ranks:
    units in decreasing cost order, each to the least loaded rank (ties: the
    lower rank, then the lower unit index).  Deterministic, so every rank
    computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(costs[i])
    for r in range(world):
        out[r].sort()
    return out


def job_seconds(local_seconds: float, torch, device=None) -> float:
    """The job's time: the maximum over the ranks of their timed-region
    seconds (all-reduce MAX), bracketed by barriers; the local value when
    no process group is initialised."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_seconds)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job time
    (weak scaling: every rank processes units_per_rank)."""
    return units_per_rank * world / seconds
