"""Partition independent problems across GPUs (ranks) by their work.

A batch of BSDE problems has no data dependencies between problems, so
several GPUs split it with no data-path collective: each rank solves its own
share.  Problems are dealt largest-first to the least-loaded rank (the LPT
rule), which keeps every share within one problem of the average work.
"""
from __future__ import annotations

import heapq


def problem_work(p: dict) -> float:
    """Node evaluations of one solve: Nx (N - k + 1) k L."""
    return float(p["Nx"]) * (int(p["N"]) - int(p["k"]) + 1) * int(p["k"]) * int(p["L"])


def shard_by_work(problems, world: int):
    """Index lists, one per rank, covering every problem exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(problems)), key=lambda i: -problem_work(problems[i]))
    heap = [(0.0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + problem_work(problems[i]), r))
    return [sorted(s) for s in shares]
