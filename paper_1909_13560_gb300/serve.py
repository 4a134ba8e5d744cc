"""Serving loop over the continuous-batching server.

Requests arrive at their (seeded) arrival times; each is admitted as soon as
the server has a free slot and enough device pool for its level ring (first
come, first served), runs while others are in flight, and is timed from its
arrival to the moment its result is collected.
"""
from __future__ import annotations

import time
from collections import deque


def serve(server, arrivals, poll_sleep: float = 0.0):
    """Run the arrivals [(t_arrival_s, problem), ...] against a started
    server in real time.  Returns per-request records and a summary."""
    pending = deque(enumerate(arrivals))
    waiting = deque()
    inflight = {}
    records = [None] * len(arrivals)
    max_inflight = 0
    t0 = time.perf_counter()
    while pending or waiting or inflight:
        now = time.perf_counter() - t0
        while pending and pending[0][1][0] <= now:
            waiting.append(pending.popleft())
        while waiting:
            i, (ta, p) = waiting[0]
            slot = server.submit(p)
            if slot is None:
                break
            inflight[slot] = (i, ta, time.perf_counter() - t0)
            waiting.popleft()
        max_inflight = max(max_inflight, len(inflight))
        for slot, res in server.poll():
            i, ta, ts = inflight.pop(slot)
            td = time.perf_counter() - t0
            records[i] = {"arrival": ta, "admitted": ts, "done": td, "latency": td - ta,
                          "result": res}
        if poll_sleep and not waiting:
            time.sleep(poll_sleep)
    t_end = time.perf_counter() - t0
    lat = sorted(r["latency"] for r in records)
    n = len(lat)
    summary = {
        "requests": n,
        "duration_s": t_end,
        "solves_per_s": n / t_end if t_end > 0 else 0.0,
        "p50_ms": 1000.0 * lat[n // 2] if n else None,
        "p99_ms": 1000.0 * lat[min(n - 1, int(0.99 * n))] if n else None,
        "max_inflight": max_inflight,
        "admit_wait_p99_ms": 1000.0 * sorted(r["admitted"] - r["arrival"] for r in records)[
            min(n - 1, int(0.99 * n))] if n else None,
    }
    return records, summary
