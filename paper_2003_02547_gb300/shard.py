"""Sharding a list of independent QPs over GPUs (one process per GPU).

QPs share nothing, so the only multi-GPU logic is host-side: split the list
by a greedy longest-processing-time rule on a per-QP cost estimate, solve
each shard on its own GPU with no data-path collective, and gather solutions
and statuses to one rank afterwards.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def qp_cost(qp) -> float:
    """Flop estimate of one Riccati factorisation of the QP:
    sum_n nx_{n+1}^2 nv + nx_{n+1} nv^2 + nv^3 / 3 + ng nv^2."""
    c = 0.0
    for n in range(qp.N + 1):
        nv = qp.nx[n] + qp.nu[n]
        nx1 = qp.nx[n + 1] if n < qp.N else 0
        c += nx1 * nx1 * nv + nx1 * nv * nv + nv ** 3 / 3.0 + qp.ng(n) * nv * nv
    return c


def lpt_shard(costs: Sequence[float], world: int) -> List[List[int]]:
    """Greedy LPT: QPs in decreasing cost go to the least loaded rank.
    Deterministic (ties broken by QP index, then rank)."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for s in shards:
        s.sort()
    return shards


def gather_results(local: dict, rank: int, world: int, dist=None):
    """Collect {qp_index: result} dicts on rank 0 (host-side, after the
    solves; None on the other ranks)."""
    if world == 1 or dist is None:
        return dict(local)
    buf = [None] * world if rank == 0 else None
    dist.gather_object(local, buf, dst=0)
    if rank != 0:
        return None
    out = {}
    for part in buf:
        out.update(part)
    return out
