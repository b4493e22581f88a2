"""Scalar CPU oracle for HalftimeHash (arXiv 2104.08865) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never loads it, and it
shares no source with the GPU library: ``halftime_ref.c`` is plain C written
from the paper, compiled with gcc into ``libhalftime_ref.so`` beside it.

Parity status: see ``halftime_ref.h`` (structural pins; absolute digests of
the full hash have no published vectors).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "halftime_ref.c")
_HDR = os.path.join(_HERE, "halftime_ref.h")
_LIB = os.path.join(_HERE, "libhalftime_ref.so")
_lock = threading.Lock()
_lib = None

WIDTHS = (16, 24, 32, 40)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2) if it is missing or stale."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.htref_seed_words.restype = ctypes.c_size_t
            L.htref_seed_words.argtypes = [ctypes.c_int]
            L.htref_seed_words_bf.restype = ctypes.c_size_t
            L.htref_seed_words_bf.argtypes = [ctypes.c_int] * 3
            L.htref_seed_expand.restype = None
            L.htref_seed_expand.argtypes = [ctypes.c_uint64, u64p, ctypes.c_size_t]
            L.htref_encode.argtypes = [ctypes.c_int, u64p, u64p]
            L.htref_ehc.argtypes = [ctypes.c_int, ctypes.c_int, u64p,
                                    ctypes.c_void_p, ctypes.c_int, u64p]
            L.htref_nh_word.restype = ctypes.c_uint64
            L.htref_nh_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.htref_hash.argtypes = [ctypes.c_int, u64p, ctypes.c_size_t,
                                     ctypes.c_void_p, ctypes.c_uint64, u64p]
            L.htref_hash_bf.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, u64p, ctypes.c_size_t,
                                        ctypes.c_void_p, ctypes.c_uint64, u64p,
                                        ctypes.POINTER(ctypes.c_int)]
            L.htref_params.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 5
            L.htref_seed_words_badger.restype = ctypes.c_size_t
            L.htref_seed_words_badger.argtypes = [ctypes.c_int, ctypes.c_int]
            L.htref_hash_badger.argtypes = [ctypes.c_int, ctypes.c_int, u64p, ctypes.c_size_t,
                                            ctypes.c_void_p, ctypes.c_uint64, u64p]
            _lib = L
    return _lib


def _u64p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _bytes_ptr(data):
    """(pointer, length, keepalive) for a bytes-like or uint8 numpy array."""
    if isinstance(data, np.ndarray):
        arr = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    else:
        arr = np.frombuffer(bytes(data), dtype=np.uint8)
    return arr.ctypes.data_as(ctypes.c_void_p), arr.size, arr


def params(width: int, b: int = 8) -> dict:
    """d, e, k, w of a width and the bytes of one execution with blocks of b words."""
    d, e, k, w, xb = (ctypes.c_int() for _ in range(5))
    rc = lib().htref_params(width, ctypes.byref(d), ctypes.byref(e), ctypes.byref(k),
                            ctypes.byref(w), ctypes.byref(xb))
    if rc:
        raise ValueError("bad width %r" % width)
    return dict(d=d.value, e=e.value, k=k.value, w=w.value, exec_bytes=8 * b * d.value * w.value)


def seed_words(width: int, b: int = 8, f: int = 8) -> int:
    return int(lib().htref_seed_words_bf(width, b, f))


def seed_expand(seed64: int, n_words: int) -> np.ndarray:
    out = np.zeros(n_words, dtype=np.uint64)
    lib().htref_seed_expand(ctypes.c_uint64(seed64 & (2**64 - 1)), _u64p(out), n_words)
    return out


def nh_word(x: int, s: int) -> int:
    return int(lib().htref_nh_word(x & (2**64 - 1), s & (2**64 - 1)))


def encode(width: int, items: np.ndarray) -> np.ndarray:
    p = params(width)
    items = np.ascontiguousarray(items, dtype=np.uint64).reshape(-1)
    assert items.size == p["d"] * p["w"]
    out = np.zeros(p["e"] * p["w"], dtype=np.uint64)
    rc = lib().htref_encode(width, _u64p(items), _u64p(out))
    assert rc == 0
    return out


def ehc(width: int, seeds: np.ndarray, exec_bytes, lane: int, b: int = 8) -> np.ndarray:
    p = params(width)
    ptr, n, keep = _bytes_ptr(exec_bytes)
    assert n >= 8 * b * p["d"] * p["w"]
    y = np.zeros(p["k"], dtype=np.uint64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    rc = lib().htref_ehc(width, b, _u64p(seeds), ptr, lane, _u64p(y))
    assert rc == 0
    return y


def hash_bytes(width: int, seeds: np.ndarray, data, *, b: int = 8, f: int = 8,
               recursive: bool = False, level_counts: bool = False):
    """Digest (numpy uint64[k]) of one string; optionally the pending-root
    counts per level of the streaming tree."""
    p = params(width)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    ptr, n, keep = _bytes_ptr(data)
    dig = np.zeros(p["k"], dtype=np.uint64)
    counts = (ctypes.c_int * 19)()
    rc = lib().htref_hash_bf(width, b, f, 1 if recursive else 0, _u64p(seeds),
                             seeds.size, ptr if n else None, n, _u64p(dig),
                             counts if level_counts else None)
    if rc:
        raise ValueError("htref_hash_bf failed: %d" % rc)
    if level_counts:
        return dig, list(counts)
    return dig


def hash_many(width: int, seeds: np.ndarray, buf: np.ndarray, offsets, lengths, b: int = 8) -> np.ndarray:
    """Digests of slices buf[offsets[i] : offsets[i]+lengths[i]] -> uint64[count, k]
    (blocks of b words: 8, or 4 for the 256-bit-block variant)."""
    p = params(width)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    buf = np.ascontiguousarray(buf).view(np.uint8).reshape(-1)
    out = np.zeros((len(lengths), p["k"]), dtype=np.uint64)
    L = lib()
    base = buf.ctypes.data
    sp = _u64p(seeds)
    for i, (o, n) in enumerate(zip(offsets, lengths)):
        o = int(o); n = int(n)
        assert o + n <= buf.size
        row = out[i]
        rc = L.htref_hash_bf(width, b, 8, 0, sp, seeds.size,
                             ctypes.c_void_p(base + o) if n else None, n,
                             row.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), None)
        if rc:
            raise ValueError("htref_hash failed: %d" % rc)
    return out


# ---- ablation: Badger's binary tree without a final NH (Section 5.2) ----------

def seed_words_badger(width: int, b: int = 8) -> int:
    """Seed words of the binary-tree ablation: E, 64 level keys per tree, R."""
    return int(lib().htref_seed_words_badger(width, b))


def hash_bytes_badger(width: int, seeds: np.ndarray, data, *, b: int = 8) -> np.ndarray:
    """Digest of one string under the binary-tree ablation (Eq. algebraic-badger
    over all EHC outputs of a tree, lane-minor; Toeplitz tail as usual)."""
    p = params(width)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    ptr, n, keep = _bytes_ptr(data)
    dig = np.zeros(p["k"], dtype=np.uint64)
    rc = lib().htref_hash_badger(width, b, _u64p(seeds), seeds.size, ptr if n else None, n, _u64p(dig))
    if rc:
        raise ValueError("htref_hash_badger failed: %d" % rc)
    return dig


def hash_many_badger(width: int, seeds: np.ndarray, buf: np.ndarray, offsets, lengths,
                     b: int = 8) -> np.ndarray:
    """Digests of slices of buf under the binary-tree ablation -> uint64[count, k]."""
    p = params(width)
    buf = np.ascontiguousarray(buf).view(np.uint8).reshape(-1)
    out = np.zeros((len(lengths), p["k"]), dtype=np.uint64)
    for i, (o, n) in enumerate(zip(offsets, lengths)):
        o = int(o); n = int(n)
        assert o + n <= buf.size
        out[i] = hash_bytes_badger(width, seeds, buf[o:o + n], b=b)
    return out
