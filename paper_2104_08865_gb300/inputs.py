"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no hash arithmetic.  It produces byte strings and length
lists only, from splitmix64 (Steele, Lea, Flood, OOPSLA 2014), written here
in its counter form: output i of a generator started at state s is
mix(s + (i+1) * 0x9E3779B97F4A7C15 mod 2^64).

Conventions:
  * the byte stream of seed s is outputs 0, 1, 2, ... in little-endian order;
  * several strings take consecutive slices of one stream;
  * log-uniform lengths in [a, b] come from a second generator seeded
    s ^ 0x4C454E: len_i = floor(exp(ln a + u_i (ln b - ln a))) with
    u_i = (x_i >> 11) * 2^-53.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
LEN_SALT = 0x4C454E

PATTERN8 = np.uint64(0x0123456789ABCDEF)


def splitmix64_words(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of splitmix64 started at state `seed`."""
    out = np.empty(count, dtype=np.uint64)
    step = 1 << 22
    s = np.uint64(seed & (2**64 - 1))
    for base in range(0, count, step):
        n = min(step, count - base)
        z = np.arange(start + base + 1, start + base + 1 + n, dtype=np.uint64)
        z *= GAMMA
        z += s
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
        out[base:base + n] = z
    return out


def _u64_to_i64(v: int) -> int:
    v &= 2**64 - 1
    return v - 2**64 if v >= 2**63 else v


def splitmix64_words_torch(seed: int, start: int, count: int, device):
    """Same outputs as splitmix64_words, computed with torch int64 ops on
    `device` (two's-complement wrap-around; logical shifts by masking)."""
    import torch
    out = torch.empty(count, dtype=torch.int64, device=device)
    step = 1 << 26
    g = _u64_to_i64(int(GAMMA))
    m1 = _u64_to_i64(int(_M1))
    m2 = _u64_to_i64(int(_M2))
    s = _u64_to_i64(seed)

    def lsr(z, n):
        return (z >> n) & ((1 << (64 - n)) - 1)

    for base in range(0, count, step):
        n = min(step, count - base)
        z = torch.arange(start + base + 1, start + base + 1 + n, dtype=torch.int64, device=device)
        z.mul_(g).add_(s)
        z.bitwise_xor_(lsr(z, 30)).mul_(m1)
        z.bitwise_xor_(lsr(z, 27)).mul_(m2)
        z.bitwise_xor_(lsr(z, 31))
        out[base:base + n] = z
    return out


def stream_bytes_torch(seed: int, offset: int, length: int, device):
    """stream_bytes as a uint8 torch tensor built on `device`."""
    import torch
    if length == 0:
        return torch.zeros(0, dtype=torch.uint8, device=device)
    w0 = offset // 8
    w1 = (offset + length + 7) // 8
    words = splitmix64_words_torch(seed, w0, w1 - w0, device)
    raw = words.view(torch.uint8)  # little-endian hosts and GPUs
    lo = offset - 8 * w0
    return raw[lo:lo + length]


def stream_bytes(seed: int, offset: int, length: int) -> np.ndarray:
    """Bytes [offset, offset+length) of the splitmix64 byte stream of `seed`."""
    if length == 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = offset // 8
    w1 = (offset + length + 7) // 8
    words = splitmix64_words(seed, w0, w1 - w0)
    raw = words.astype("<u8").view(np.uint8)
    lo = offset - 8 * w0
    return raw[lo:lo + length].copy()


def log_uniform_lengths(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """`count` lengths, log-uniform in [lo, hi] (int64)."""
    x = splitmix64_words(seed ^ LEN_SALT, 0, count)
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    ln_a, ln_b = np.log(float(lo)), np.log(float(hi))
    n = np.floor(np.exp(ln_a + u * (ln_b - ln_a))).astype(np.int64)
    return np.clip(n, lo, hi)


def pattern_bytes(kind: str, length: int, seed: int = 5) -> np.ndarray:
    """Content classes of the edge sweep: zero, ff, pattern8, random."""
    if kind == "zero":
        return np.zeros(length, dtype=np.uint8)
    if kind == "ff":
        return np.full(length, 0xFF, dtype=np.uint8)
    if kind == "pattern8":
        reps = (length + 7) // 8
        return np.full(reps, PATTERN8, dtype="<u8").view(np.uint8)[:length].copy()
    if kind == "random":
        return stream_bytes(seed, 0, length)
    raise ValueError(kind)


def packed_batch(seed: int, lengths, align: int = 256):
    """Consecutive slices of one stream, each placed at an `align`-byte aligned
    offset of one buffer.  Returns (buffer uint8, offsets int64)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    slots = (lengths + align - 1) // align * align
    offsets = np.concatenate([[0], np.cumsum(slots)[:-1]]).astype(np.int64)
    total = int(slots.sum()) if len(lengths) else 0
    buf = np.zeros(max(total, align), dtype=np.uint8)
    stream = stream_bytes(seed, 0, int(lengths.sum()))
    for s, o, n in zip(starts, offsets, lengths):
        buf[o:o + n] = stream[s:s + n]
    return buf, offsets
