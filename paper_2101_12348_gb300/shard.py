"""Sharding of periodogram work across processes, one GPU each.

The path has no exchange step: lightcurves are independent, the templates of
a bank only share the (cheap) sums of their curve, and frequencies are
independent given the sums.  So a multi-GPU run is a partition of the work
units, one part per rank, with no collective on the data path; the only
communication is the host-level merge of per-rank results at the end.

  partition_by_cost  curves of a survey, balanced by an estimated cost per
                     curve (N_obs * N_f or similar): longest-processing-time
                     first, each curve to the least-loaded rank;
  partition_strided  templates of a bank: rank r takes r, r + world, ...;
  merge_parts        per-rank (indices, rows) pairs back into one array in
                     the single-GPU order, checking that the parts are
                     disjoint and cover every index;
  gather_to_root     a picklable object from every rank to rank 0 over the
                     run's process group (outside any timed region).
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_by_cost(costs, world: int) -> list:
    """Indices of the units each rank takes, balanced by cost (greedy LPT).
    Every part is sorted ascending; parts are disjoint and cover 0..n-1."""
    costs = np.asarray(costs, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if np.any(~np.isfinite(costs)) or np.any(costs < 0):
        raise ValueError("costs must be finite and non-negative")
    order = np.argsort(-costs, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def partition_strided(n: int, world: int) -> list:
    """Rank r takes units r, r + world, r + 2 world, ... of n."""
    if world < 1:
        raise ValueError("world must be >= 1")
    return [np.arange(r, n, world, dtype=np.int64) for r in range(world)]


def part_loads(costs, parts) -> np.ndarray:
    costs = np.asarray(costs, dtype=np.float64)
    return np.array([float(costs[p].sum()) for p in parts])


def merge_parts(n: int, parts) -> np.ndarray:
    """parts: sequence of (indices, rows) with rows[j] the result of unit
    indices[j] (rows may be 1-D or have trailing dimensions).  Returns the
    n results in unit order; raises if the parts overlap or miss a unit."""
    parts = [(np.asarray(i, dtype=np.int64), np.asarray(v)) for i, v in parts]
    seen = np.zeros(n, dtype=bool)
    out = None
    for idx, rows in parts:
        if rows.shape[0] != idx.shape[0]:
            raise ValueError("each part needs one row per index")
        if idx.size and (idx.min() < 0 or idx.max() >= n):
            raise ValueError("index out of range")
        if np.any(seen[idx]) or np.unique(idx).size != idx.size:
            raise ValueError("parts overlap")
        seen[idx] = True
        if out is None:
            out = np.empty((n,) + rows.shape[1:], dtype=rows.dtype)
        out[idx] = rows
    if not np.all(seen):
        raise ValueError(f"parts miss {int(np.count_nonzero(~seen))} unit(s)")
    if out is None:
        out = np.empty((n,))
    return out


def gather_to_root(pg, obj, rank: int, world: int):
    """List of every rank's `obj` on rank 0 (None elsewhere); pg is
    torch.distributed or None for a single process."""
    if pg is None or world == 1:
        return [obj]
    out = [None] * world if rank == 0 else None
    pg.gather_object(obj, out, dst=0)
    return out
