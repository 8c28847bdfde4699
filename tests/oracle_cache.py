"""Oracle values on seeded destination points, computed once per test session
and shared by the GPU test files that compare against the same workload."""
from __future__ import annotations

import functools

import oracle
from paper_1203_3583_gb300 import workloads as W


@functools.lru_cache(maxsize=None)
def sampled(name: str, count: int, seed: int):
    """(g, u1, d1, pts, eq7 at pts) for a standard workload."""
    g, u1, d1 = W.make(name)
    pts = W.sample_points(g, count, seed=seed)
    return g, u1, d1, pts, oracle.eq7(g, u1, d1, points=pts)
