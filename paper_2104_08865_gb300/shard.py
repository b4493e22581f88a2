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


def part_bounds(total_len: int, granule: int, world: int):
    """Byte boundaries of `world` parts of one string: multiples of the
    granule, about equal, the last one ending at total_len."""
    units = -(-total_len // granule) if total_len else 0
    b = [min(total_len, (units * r // world) * granule) for r in range(world)] + [total_len]
    return b


def hash_split(hasher, data, total_len: int, world: int, rank: int, device=None):
    """Hashes one string split across the ranks of the process group: rank r
    hashes part r of `data` (a CUDA uint8 tensor holding the whole string,
    or at least part r at its offset) into a state tensor, the states are
    summed with one all-reduce, and every rank finishes the same digest.
    Returns the digest as a uint64 numpy array."""
    import torch
    import torch.distributed as dist

    from . import abi
    dev = device if device is not None else data.device
    words = abi.ht_part_state_words(hasher.ctx, total_len)
    state = torch.zeros(words, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    abi.ht_part_begin(hasher.ctx, total_len, state.data_ptr(), words, stream)
    b = part_bounds(total_len, abi.ht_part_granule(hasher.ctx), world)
    lo, hi = b[rank], b[rank + 1]
    if hi > lo or hi == total_len:
        abi.ht_hash_part(hasher.ctx, data.data_ptr() + lo, lo, hi - lo, stream)
    torch.cuda.synchronize(dev)
    if dist.is_available() and dist.is_initialized() and world > 1:
        dist.all_reduce(state, op=dist.ReduceOp.SUM)  # int64 sums wrap like uint64
    out = torch.empty(hasher.k, dtype=torch.int64, device=dev)
    abi.ht_finish_parts(hasher.ctx, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy().view(np.uint64)
