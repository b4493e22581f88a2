"""HalftimeHash composed with a short-input hash family -- test infrastructure.

Only the tests and the CPU legs of the benchmark import this module; the GPU
library never loads it and shares no code with it.

The paper presents HalftimeHash as a "universe collapsing" family (Section 1):
it maps long strings to short digests, and a family made for short inputs can
then treat the digests as if they were the strings; almost universality
composes, with the two collision bounds adding up (the composition lemma of
Section 5.2).  The GPU table keys long strings by their digests this way.
This module states what it computes, in plain Python integers:

* ``slot_hash``: vector multiply-shift over the digest's 32-bit halves,
  ``(a_0 + sum_i a_{i+1} * x_i) mod 2^64``, of which the table uses the top
  bits (Dietzfelbinger, Hagerup, Katajainen and Penttonen, J. Algorithms
  1997; the vector form as in Thorup, "High speed hashing for integers and
  strings", 2015: with 32-bit x_i and uniform 64-bit a_i the top l <= 33
  bits are strongly universal).  The keys a_0..a_2k are splitmix64 outputs
  of the table's seed (the same counter-based generator as the hash seeds).
* ``representatives``: entry ids number digests in insertion order; the
  representative of entry i is the smallest id whose digest equals its own.
* ``find``: the smallest entry id whose digest equals a query, else
  0xffffffff.

Parity: ``slot_hash`` is pinned by closed forms and by the strong
universality of its top bits (tests/test_compose_cpu.py);
``representatives`` and ``find`` are their plain definitions.
"""
from __future__ import annotations

import numpy as np

from . import seed_expand

MASK64 = (1 << 64) - 1
NOT_FOUND = 0xFFFFFFFF


def table_keys(seed64: int, k: int) -> list:
    """The 2k + 1 multiply-shift keys of a table over k-word digests."""
    return [int(v) for v in seed_expand(seed64, 2 * k + 1)]


def slot_hash(keys, digest) -> int:
    """(a_0 + sum over the digest's 32-bit halves x_i of a_{i+1} x_i) mod 2^64,
    halves in order: low then high half of word 0, then of word 1, ..."""
    h = int(keys[0])
    for i, w in enumerate(digest):
        w = int(w)
        h += int(keys[1 + 2 * i]) * (w & 0xFFFFFFFF) + int(keys[2 + 2 * i]) * (w >> 32)
    return h & MASK64


def representatives(digests, first_id: int = 0, earlier=None) -> np.ndarray:
    """rep[i] for digests (rows) inserted as ids first_id, first_id + 1, ...;
    `earlier` maps digest tuples of entries inserted before to their ids
    (updated in place)."""
    seen = {} if earlier is None else earlier
    out = np.empty(len(digests), dtype=np.uint32)
    for i, d in enumerate(digests):
        key = tuple(int(v) for v in d)
        if key not in seen:
            seen[key] = first_id + i
        out[i] = seen[key]
    return out


def find(digests, table: dict) -> np.ndarray:
    """The id of the entry equal to each query digest, else 0xffffffff."""
    return np.array([table.get(tuple(int(v) for v in d), NOT_FOUND) for d in digests], dtype=np.uint32)
