"""Host-side multi-process logic (one process per GPU).

The single-LP path has no data-parallel exchange: under torchrun every rank
runs its own replica and the job's throughput is the units all ranks
processed divided by the slowest rank's time.  A batch of independent LPs
shards by problem: each rank solves its own subset (no collective on the
data path; only the final timing/result reduction).  Everything here is
backend-agnostic torch.distributed (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_by_weight(weights, world: int, rank: int) -> list:
    """Indices of the items rank `rank` of `world` takes: longest-processing-
    time-first greedy (heaviest item to the least loaded rank, ties to the
    lower rank), deterministic, each item exactly once.  Returned ascending."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    w = np.asarray(weights, dtype=np.float64)
    order = np.lexsort((np.arange(w.shape[0]), -w))  # heaviest first, then by index
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(int(i))
        heapq.heappush(heap, (load + float(w[i]), r))
    return sorted(mine)


def _is_dist():
    import torch.distributed as dist

    return dist.is_available() and dist.is_initialized()


def reduce_scalar(value: float, op: str, device=None) -> float:
    """All-reduce one number over the ranks ('max' or 'sum'); identity when
    torch.distributed is not initialized."""
    if not _is_dist():
        return float(value)
    import torch
    import torch.distributed as dist

    if device is None and dist.get_backend() == "nccl":
        device = "cuda"  # NCCL reduces device tensors only
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def job_throughput(local_units: float, local_seconds: float, device=None):
    """(units of all ranks / max seconds over ranks, max seconds): the
    whole-job rate of replicas or shards timed between two barriers."""
    total = reduce_scalar(local_units, "sum", device)
    slowest = reduce_scalar(local_seconds, "max", device)
    return total / slowest, slowest
