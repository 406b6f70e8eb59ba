"""Replicas on several GPUs (one process per GPU): the path shards into
independent units (GEMMs of the benchmark, systems of a batch, requests of a
serving stream), so no collective touches the data.  Two pieces of host
logic are shared by the ranks:

* ``partition_by_cost``: a deterministic assignment of independent units to
  ranks, longest first onto the least-loaded rank (LPT).  Every rank computes
  the same assignment from the same inputs, so the router needs no exchange.
* ``max_over_ranks``: the one reduction of a timed run, the slowest rank's
  time, through whatever process group the caller has (NCCL on GPUs, gloo on
  CPUs).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def partition_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the units each rank takes: units in decreasing cost (ties by
    index), each onto the rank with the least total so far (ties by rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for lst in out:
        lst.sort()
    return out


def solve_cost(n: int, nrhs: int = 1) -> float:
    """Work estimate of one LU + refinement solve: 2/3 n^3 + refinement n^2 nrhs."""
    return 2.0 / 3.0 * n ** 3 + 10.0 * n * n * nrhs


def rank_share(costs: Sequence[float], rank: int, world: int) -> List[int]:
    return partition_by_cost(costs, world)[rank]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over the ranks of the default process group (the
    value itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
