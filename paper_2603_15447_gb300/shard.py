"""Partition a batch of curves over ranks (one process per GPU).

Curves are independent, so a batch shards into contiguous curve ranges with no
exchange between ranks during evaluation.  Ranges are balanced by the number
of samples (the work) rather than the number of curves: rank r takes the
curves whose cumulative sample count falls in [r W / N, (r+1) W / N) of the
total W.
"""
from __future__ import annotations

import numpy as np


def balanced_ranges(n_samples, world: int):
    """Contiguous [start, stop) curve ranges, one per rank, balanced by the
    prefix sum of ``n_samples`` (per-curve sample counts)."""
    n_samples = np.asarray(n_samples, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(n_samples.sum())
    csum = np.concatenate([[0], np.cumsum(n_samples)])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        bounds.append(int(np.searchsorted(csum, target, side="left")))
    bounds.append(len(n_samples))
    bounds = np.maximum.accumulate(np.array(bounds))
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def shard_of(n_samples, rank: int, world: int):
    """The [start, stop) curve range of ``rank``."""
    return balanced_ranges(n_samples, world)[rank]
