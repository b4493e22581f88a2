"""Splitting a batch of strings across ranks (one process per GPU).

Strings are independent, so a batch shards with no data-path collective:
each rank hashes a contiguous run of strings holding about 1/world of the
bytes, and the digests are gathered once at the end (a few bytes per string).
These helpers are host logic only; the hashing itself is the CUDA library's.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(lengths, world: int):
    """Boundaries b[0..world] such that rank r takes strings [b[r], b[r+1]):
    contiguous runs with about equal byte totals (each string counted as at
    least one byte so empty strings spread too)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lens = np.maximum(np.asarray(lengths, dtype=np.int64), 1)
    csum = np.concatenate([[0], np.cumsum(lens)])
    total = int(csum[-1])
    targets = [total * r // world for r in range(world + 1)]
    b = np.searchsorted(csum, targets, side="left").astype(np.int64)
    b[0], b[-1] = 0, len(lens)
    return np.maximum.accumulate(np.minimum(b, len(lens)))


def shard_of(lengths, world: int, rank: int):
    """Index range (lo, hi) of the strings of `rank`."""
    b = shard_bounds(lengths, world)
    return int(b[rank]), int(b[rank + 1])


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float (e.g. a time) over the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_digests(local: np.ndarray, counts, device=None) -> np.ndarray:
    """Concatenates every rank's uint64 digest rows (rank order).  `counts`
    holds each rank's number of rows; every rank returns the full array."""
    import torch
    import torch.distributed as dist
    local = np.ascontiguousarray(local, dtype=np.uint64)
    if not dist.is_available() or not dist.is_initialized():
        return local
    k = local.shape[1]
    width = max(int(c) for c in counts)
    buf = np.zeros((width, k), dtype=np.uint64)
    buf[:local.shape[0]] = local
    t = torch.from_numpy(buf.view(np.int64)).to(device) if device is not None else torch.from_numpy(buf.view(np.int64))
    parts = [torch.empty_like(t) for _ in counts]
    dist.all_gather(parts, t)
    rows = [p.cpu().numpy().view(np.uint64)[:int(c)] for p, c in zip(parts, counts)]
    return np.concatenate(rows, axis=0)
