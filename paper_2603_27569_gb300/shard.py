"""Sharding a batch of transforms over ranks (one process per GPU).

Transforms are independent, so a batch splits across GPUs with no exchange
on the data path: every rank transforms its own rows with its own plan and
only the timing is reduced (max over ranks).

  shard_rows(batch, rank, world)  contiguous, sizes differing by at most 1.
  shard_ragged(N, world)          per-transform rank for a mixed-length list,
                                  balanced by the nominal work 5 N log2 N
                                  (longest-processing-time first, ties by
                                  index, so every rank computes the same map).
  max_over_ranks(x)               the largest value over the process group
                                  (timing only; identity without a group).
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def shard_rows(batch: int, rank: int, world: int) -> tuple[int, int]:
    """(first row, row count) of `rank`'s share of `batch` rows."""
    if world < 1 or not 0 <= rank < world or batch < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(batch, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def transform_cost(N) -> np.ndarray:
    N = np.asarray(N, dtype=np.float64)
    return 5.0 * N * np.log2(N)


def shard_ragged(N, world: int) -> np.ndarray:
    """Rank of every transform (int32), LPT-balanced by 5 N log2 N."""
    N = np.asarray(N)
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = transform_cost(N)
    order = sorted(range(len(N)), key=lambda i: (-cost[i], i))
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(N), dtype=np.int32)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + float(cost[i]), r))
    return owner


def max_over_ranks(value: float) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
