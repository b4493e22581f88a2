"""Thin ctypes binding of libhalftime (include/halftime.h): same names, argument
marshalling only.  Every hash is computed by the CUDA library; there is no
Python or CPU fallback: if the library is missing, importing this module
raises.

Pointers may be given as ints or as torch tensors (their data_ptr()); streams
as ints, torch.cuda.Stream objects or None (the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HALFTIME_CHECKED=1 loads the checked build (every kernel access
# range-checked; same entry points) instead of the product library
CHECKED = os.environ.get("HALFTIME_CHECKED", "") == "1"
LIB_PATH = os.path.join(_HERE, "libhalftime_check.so" if CHECKED else "libhalftime.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libhalftime.so is not built: run `python -c \"import __graft_entry__ as g; "
                      "g.build()\"` (or paper_2104_08865_gb300/build.py)")

_lib = ctypes.CDLL(LIB_PATH)

HT_OK = 0
HT_ERR_ARG = -1
HT_ERR_WIDTH = -2
HT_ERR_TOO_LONG = -3
HT_ERR_CUDA = -4
HT_ERR_NOMEM = -5
HT_ERR_BUDGET = -6
HT_ERR_TIMEOUT = -7
HT_ERR_BUSY = -8
HT_ERR_DEVICE = -9
WIDTHS = (16, 24, 32, 40)
# width_bytes | HT_BLOCK_256 selects blocks of 4 words (256 bits) instead of 8
HT_BLOCK_256 = 0x100
# width_bytes | HT_TREE_BINARY selects the binary-tree ablation (Badger's tree, no final NH)
HT_TREE_BINARY = 0x200
HT_BUILD_CHECKED = 1


class HalftimeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class ht_shape(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("chunk_levels", ctypes.c_int), ("stages", ctypes.c_int),
                ("threads_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int)]


class ht_server_opts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("max_batch", ctypes.c_size_t),
                ("max_queue", ctypes.c_size_t), ("max_wait_us", ctypes.c_uint64),
                ("pinned_mode", ctypes.c_int)]


class ht_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("bytes_completed", ctypes.c_uint64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("wall_s", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u64p = ctypes.POINTER(ctypes.c_uint64)
_int = ctypes.c_int
_sz = ctypes.c_size_t

_PROTOS = {
    "ht_last_error": (_int, [ctypes.c_char_p, _sz]),
    "ht_seed_words": (_sz, [_int]),
    "ht_seed_expand": (_int, [_u64, _int, _u64p, _sz]),
    "ht_ctx_create": (_int, [_int, _u64p, _sz, _vp, ctypes.POINTER(_vp)]),
    "ht_ctx_destroy": (_int, [_vp]),
    "ht_ctx_reserve": (_int, [_vp, _u64, _sz]),
    "ht_ctx_rekey": (_int, [_vp, _u64p, _sz, _vp]),
    "ht_ctx_status": (_int, [_vp, _vp]),
    "ht_ctx_set_flags": (_int, [_vp, ctypes.c_uint]),
    "ht_hash": (_int, [_vp, _vp, _u64, _vp, _vp]),
    "ht_hash_host": (_int, [_vp, _vp, _u64, _vp, _vp]),
    "ht_hash_batch": (_int, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "ht_hash_batch_naive": (_int, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "ht_hash_noalloc": (_int, [_int, _u64p, _sz, _vp, _u64, _vp, _vp]),
    "ht_inc_create": (_int, [_vp, ctypes.POINTER(_vp)]),
    "ht_inc_destroy": (_int, [_vp]),
    "ht_inc_init": (_int, [_vp, _vp]),
    "ht_inc_update": (_int, [_vp, _vp, _u64, _vp]),
    "ht_inc_update_host": (_int, [_vp, _vp, _u64, _vp]),
    "ht_inc_final": (_int, [_vp, _vp, _vp]),
    "ht_inc_length": (_u64, [_vp]),
    "ht_inc_granule": (_u64, [_vp]),
    "ht_inc_state_bytes": (_sz, [_vp]),
    "ht_inc_export": (_int, [_vp, _vp, _sz, _vp]),
    "ht_inc_import": (_int, [_vp, _vp, _sz, _vp]),
    "ht_short_hash_keys": (_int, [_u64, _int, _u64p, _sz]),
    "ht_short_hash": (_int, [_u64p, _int, _u64p, _u64p]),
    "ht_table_create": (_int, [_vp, _u64, _u64, ctypes.POINTER(_vp)]),
    "ht_table_destroy": (_int, [_vp]),
    "ht_table_clear": (_int, [_vp, _vp]),
    "ht_table_entries": (_u64, [_vp]),
    "ht_table_slot_bits": (_int, [_vp]),
    "ht_table_keys": (_int, [_vp, _u64p, _sz]),
    "ht_table_insert": (_int, [_vp, _vp, _sz, _vp, _vp]),
    "ht_table_find": (_int, [_vp, _vp, _sz, _vp, _vp]),
    "ht_table_status": (_int, [_vp, _vp]),
    "ht_part_granule": (_u64, [_vp]),
    "ht_part_state_words": (_sz, [_vp, _u64]),
    "ht_part_begin": (_int, [_vp, _u64, _vp, _sz, _vp]),
    "ht_hash_part": (_int, [_vp, _vp, _u64, _u64, _vp]),
    "ht_part_state": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_sz)]),
    "ht_part_merge": (_int, [_vp, _vp, _sz, _vp]),
    "ht_finish_parts": (_int, [_vp, _vp, _vp]),
    "ht_autotune": (_int, [_vp, _u64, _vp, ctypes.POINTER(ht_shape)]),
    "ht_autotune_batch": (_int, [_vp, _vp, _vp, _sz, _vp, _vp, ctypes.POINTER(ht_shape)]),
    "ht_get_shape": (_int, [_vp, _u64, ctypes.POINTER(ht_shape)]),
    "ht_set_shape": (_int, [_vp, _u64, ctypes.POINTER(ht_shape)]),
    "ht_ctx_launches": (_u64, [_vp]),
    "ht_build_flags": (ctypes.c_uint, []),
    "ht_check_probe": (_int, [_vp, _u64, _u64, _vp]),
    "ht_wait_probe": (_int, [_vp, _u64, _vp]),
    "ht_testing_set_wait_cycles": (_int, [_vp, _u64]),
    "ht_inc_status": (_int, [_vp, _vp]),
    "ht_server_create": (_int, [_vp, _u64, ctypes.POINTER(ht_server_opts), ctypes.POINTER(_vp)]),
    "ht_server_create_fake": (_int, [_int, _u64, ctypes.POINTER(ht_server_opts), _u64,
                                     ctypes.c_int64, ctypes.POINTER(_vp)]),
    "ht_server_submit": (_int, [_vp, _vp, _u64, _int, _vp, _u64p]),
    "ht_server_poll": (_int, [_vp, _u64, ctypes.POINTER(_int)]),
    "ht_server_wait": (_int, [_vp, _u64, _u64]),
    "ht_server_cancel": (_int, [_vp, _u64]),
    "ht_server_drain": (_int, [_vp, _u64]),
    "ht_server_replay": (_int, [_vp, _vp, _vp, _vp, _vp, _sz, _vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "ht_server_stats": (_int, [_vp, ctypes.POINTER(ht_server_stats_t), _int]),
    "ht_server_latencies": (_sz, [_vp, ctypes.POINTER(ctypes.c_double), _sz]),
    "ht_server_destroy": (_int, [_vp]),
}

for _name, (_res, _args) in _PROTOS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols():
    """Names of the C-ABI entry points this binding declares."""
    return sorted(_PROTOS)


def lib():
    return _lib


# ---- marshalling -------------------------------------------------------------

def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a pointer, tensor or array, got %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s or None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or None
    raise TypeError("expected a stream, got %r" % type(s))


def _check(rc):
    if rc != HT_OK:
        buf = ctypes.create_string_buffer(256)
        _lib.ht_last_error(buf, 256)
        raise HalftimeError(rc, buf.value.decode(errors="replace"))
    return rc


# ---- C-ABI names ---------------------------------------------------------------

def ht_last_error():
    buf = ctypes.create_string_buffer(256)
    code = _lib.ht_last_error(buf, 256)
    return code, buf.value.decode(errors="replace")


def ht_seed_words(width: int) -> int:
    return int(_lib.ht_seed_words(width))


def ht_seed_expand(seed64: int, width: int) -> np.ndarray:
    n = ht_seed_words(width)
    if n == 0:
        raise HalftimeError(HT_ERR_WIDTH, "unsupported width %r" % width)
    out = np.zeros(n, dtype=np.uint64)
    _check(_lib.ht_seed_expand(seed64 & (2**64 - 1), width,
                               out.ctypes.data_as(_u64p), n))
    return out


def ht_ctx_create(width: int, seed_words, stream=None) -> int:
    seed_words = np.ascontiguousarray(seed_words, dtype=np.uint64)
    out = _vp()
    _check(_lib.ht_ctx_create(width, seed_words.ctypes.data_as(_u64p), seed_words.size,
                              _stream(stream), ctypes.byref(out)))
    return out.value


def ht_ctx_destroy(ctx: int) -> None:
    _check(_lib.ht_ctx_destroy(ctx))


def ht_ctx_rekey(ctx: int, seed_words, stream=None) -> None:
    seed_words = np.ascontiguousarray(seed_words, dtype=np.uint64)
    _check(_lib.ht_ctx_rekey(ctx, seed_words.ctypes.data_as(_u64p), seed_words.size,
                             _stream(stream)))


def ht_ctx_reserve(ctx: int, max_total_bytes: int, max_strings: int) -> None:
    _check(_lib.ht_ctx_reserve(ctx, max_total_bytes, max_strings))


HT_FLAG_OVERLAP_LAUNCHES = 1


def ht_ctx_set_flags(ctx: int, flags: int) -> None:
    _check(_lib.ht_ctx_set_flags(ctx, flags))


def ht_ctx_status(ctx: int, stream=None) -> None:
    _check(_lib.ht_ctx_status(ctx, _stream(stream)))


def ht_hash(ctx: int, data_dev, length: int, digest_dev, stream=None) -> None:
    _check(_lib.ht_hash(ctx, _ptr(data_dev), length, _ptr(digest_dev), _stream(stream)))


def ht_hash_host(ctx: int, data_host, length: int, digest_host, stream=None) -> None:
    _check(_lib.ht_hash_host(ctx, _ptr(data_host), length, _ptr(digest_host), _stream(stream)))


def ht_hash_batch(ctx: int, ptrs_dev, lens_dev, count: int, digests_dev, stream=None) -> None:
    _check(_lib.ht_hash_batch(ctx, _ptr(ptrs_dev), _ptr(lens_dev), count, _ptr(digests_dev),
                              _stream(stream)))


def ht_hash_batch_naive(ctx: int, ptrs_host, lens_host, count: int, digests_dev,
                        stream=None) -> None:
    _check(_lib.ht_hash_batch_naive(ctx, _ptr(ptrs_host), _ptr(lens_host), count,
                                    _ptr(digests_dev), _stream(stream)))


def ht_hash_noalloc(width: int, seed_words, data_dev, length: int, digest_dev, stream=None) -> None:
    """Hash without any allocation (scratch in the library's fixed device array)."""
    seed_words = np.ascontiguousarray(seed_words, dtype=np.uint64)
    _check(_lib.ht_hash_noalloc(width, seed_words.ctypes.data_as(_u64p), seed_words.size,
                                _ptr(data_dev), length, _ptr(digest_dev), _stream(stream)))


def ht_inc_create(ctx: int) -> int:
    h = _vp()
    _check(_lib.ht_inc_create(ctx, ctypes.byref(h)))
    return h.value


def ht_inc_destroy(h: int) -> None:
    _check(_lib.ht_inc_destroy(h))


def ht_inc_init(h: int, stream=None) -> None:
    _check(_lib.ht_inc_init(h, _stream(stream)))


def ht_inc_update(h: int, data_dev, length: int, stream=None) -> None:
    _check(_lib.ht_inc_update(h, _ptr(data_dev), length, _stream(stream)))


def ht_inc_update_host(h: int, data_host, length: int, stream=None) -> None:
    _check(_lib.ht_inc_update_host(h, _ptr(data_host), length, _stream(stream)))


def ht_inc_final(h: int, digest_dev, stream=None) -> None:
    _check(_lib.ht_inc_final(h, _ptr(digest_dev), _stream(stream)))


def ht_inc_status(h: int, stream=None) -> None:
    _check(_lib.ht_inc_status(h, _stream(stream)))


def ht_inc_length(h: int) -> int:
    return int(_lib.ht_inc_length(h))


def ht_inc_granule(h: int) -> int:
    return int(_lib.ht_inc_granule(h))


def ht_inc_state_bytes(h: int) -> int:
    return int(_lib.ht_inc_state_bytes(h))


def ht_inc_export(h: int, stream=None) -> bytes:
    """The open string's saved state (host bytes)."""
    buf = ctypes.create_string_buffer(ht_inc_state_bytes(h))
    _check(_lib.ht_inc_export(h, buf, len(buf), _stream(stream)))
    return buf.raw


def ht_inc_import(h: int, state: bytes, stream=None) -> None:
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(_lib.ht_inc_import(h, buf, len(state), _stream(stream)))


def ht_short_hash_keys(seed64: int, width: int) -> np.ndarray:
    out = np.zeros(2 * ((width & 0xFF) // 8) + 1, dtype=np.uint64)
    _check(_lib.ht_short_hash_keys(seed64, width, out.ctypes.data_as(_u64p), out.size))
    return out


def ht_short_hash(keys, width: int, digest) -> int:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    digest = np.ascontiguousarray(digest, dtype=np.uint64)
    out = ctypes.c_uint64()
    _check(_lib.ht_short_hash(keys.ctypes.data_as(_u64p), width, digest.ctypes.data_as(_u64p),
                              ctypes.byref(out)))
    return out.value


def ht_table_create(ctx: int, max_entries: int, seed64: int) -> int:
    t = _vp()
    _check(_lib.ht_table_create(ctx, max_entries, seed64, ctypes.byref(t)))
    return t.value


def ht_table_destroy(t: int) -> None:
    _check(_lib.ht_table_destroy(t))


def ht_table_clear(t: int, stream=None) -> None:
    _check(_lib.ht_table_clear(t, _stream(stream)))


def ht_table_entries(t: int) -> int:
    return int(_lib.ht_table_entries(t))


def ht_table_slot_bits(t: int) -> int:
    return int(_lib.ht_table_slot_bits(t))


def ht_table_keys(t: int, width: int) -> np.ndarray:
    out = np.zeros(2 * ((width & 0xFF) // 8) + 1, dtype=np.uint64)
    _check(_lib.ht_table_keys(t, out.ctypes.data_as(_u64p), out.size))
    return out


def ht_table_insert(t: int, digests_dev, count: int, rep_dev=None, stream=None) -> None:
    _check(_lib.ht_table_insert(t, _ptr(digests_dev), count, _ptr(rep_dev), _stream(stream)))


def ht_table_find(t: int, digests_dev, count: int, found_dev, stream=None) -> None:
    _check(_lib.ht_table_find(t, _ptr(digests_dev), count, _ptr(found_dev), _stream(stream)))


def ht_table_status(t: int, stream=None) -> None:
    _check(_lib.ht_table_status(t, _stream(stream)))


def ht_part_granule(ctx: int) -> int:
    return int(_lib.ht_part_granule(ctx))


def ht_part_state_words(ctx: int, total_len: int) -> int:
    return int(_lib.ht_part_state_words(ctx, total_len))


def ht_part_begin(ctx: int, total_len: int, state_dev=None, words: int = 0, stream=None) -> None:
    _check(_lib.ht_part_begin(ctx, total_len, _ptr(state_dev), words, _stream(stream)))


def ht_hash_part(ctx: int, part_dev, part_offset: int, part_len: int, stream=None) -> None:
    _check(_lib.ht_hash_part(ctx, _ptr(part_dev), part_offset, part_len, _stream(stream)))


def ht_part_state(ctx: int):
    """(device pointer, words) of the open part state."""
    p = _vp()
    n = _sz()
    _check(_lib.ht_part_state(ctx, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def ht_part_merge(ctx: int, state_dev, words: int, stream=None) -> None:
    _check(_lib.ht_part_merge(ctx, _ptr(state_dev), words, _stream(stream)))


def ht_finish_parts(ctx: int, digest_dev, stream=None) -> None:
    _check(_lib.ht_finish_parts(ctx, _ptr(digest_dev), _stream(stream)))


def ht_autotune(ctx: int, length: int, stream=None) -> dict:
    best = ht_shape()
    _check(_lib.ht_autotune(ctx, length, _stream(stream), ctypes.byref(best)))
    return {n: getattr(best, n) for n, _ in ht_shape._fields_}


def ht_autotune_batch(ctx: int, ptrs_dev, lens_dev, count: int, digests_dev, stream=None) -> dict:
    """Times the candidate batch shapes on this batch; keeps the fastest."""
    best = ht_shape()
    _check(_lib.ht_autotune_batch(ctx, _ptr(ptrs_dev), _ptr(lens_dev), count, _ptr(digests_dev),
                                  _stream(stream), ctypes.byref(best)))
    return {n: getattr(best, n) for n, _ in ht_shape._fields_}


def ht_get_shape(ctx: int, length: int) -> dict:
    s = ht_shape()
    _check(_lib.ht_get_shape(ctx, length, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in ht_shape._fields_}


def ht_set_shape(ctx: int, length: int, kernel: int = 0, chunk_levels: int = 2, stages: int = 3,
                 threads_per_block: int = 192, blocks_per_sm: int = 1) -> None:
    s = ht_shape(kernel, chunk_levels, stages, threads_per_block, blocks_per_sm)
    _check(_lib.ht_set_shape(ctx, length, ctypes.byref(s)))


def ht_ctx_launches(ctx: int) -> int:
    return int(_lib.ht_ctx_launches(ctx))


def ht_build_flags() -> int:
    """HT_BUILD_CHECKED for the checked build, else 0."""
    return int(_lib.ht_build_flags())


def ht_wait_probe(ctx: int, cycles: int, stream=None) -> None:
    _check(_lib.ht_wait_probe(ctx, cycles, _stream(stream)))


def ht_testing_set_wait_cycles(ctx: int, cycles: int) -> None:
    """Testing: limit of the stream kernel's stage waits on this context (0: default)."""
    _check(_lib.ht_testing_set_wait_cycles(ctx, cycles))


def ht_check_probe(ctx: int, index: int, limit: int, stream=None) -> None:
    _check(_lib.ht_check_probe(ctx, index, limit, _stream(stream)))


def _opts(n_streams=0, max_batch=0, max_queue=0, max_wait_us=0, pinned_mode=0):
    return ht_server_opts(n_streams, max_batch, max_queue, max_wait_us, pinned_mode)


def ht_server_create(ctx: int, budget_bytes: int, **opts) -> int:
    out = _vp()
    o = _opts(**opts)
    _check(_lib.ht_server_create(ctx, budget_bytes, ctypes.byref(o), ctypes.byref(out)))
    return out.value


def ht_server_create_fake(width: int, budget_bytes: int, batch_delay_us: int = 0,
                          fail_batch: int = -1, **opts) -> int:
    out = _vp()
    o = _opts(**opts)
    _check(_lib.ht_server_create_fake(width, budget_bytes, ctypes.byref(o), batch_delay_us,
                                      fail_batch, ctypes.byref(out)))
    return out.value


def ht_server_submit(srv: int, ptr, length: int, ptr_is_host_pinned: bool, digest_host) -> int:
    t = ctypes.c_uint64()
    _check(_lib.ht_server_submit(srv, _ptr(ptr), length, 1 if ptr_is_host_pinned else 0,
                                 _ptr(digest_host), ctypes.byref(t)))
    return t.value


def ht_server_poll(srv: int, ticket: int) -> bool:
    done = _int()
    _check(_lib.ht_server_poll(srv, ticket, ctypes.byref(done)))
    return bool(done.value)


def ht_server_wait(srv: int, ticket: int, timeout_us: int) -> None:
    _check(_lib.ht_server_wait(srv, ticket, timeout_us))


def ht_server_cancel(srv: int, ticket: int) -> None:
    _check(_lib.ht_server_cancel(srv, ticket))


def ht_server_replay(srv: int, ptrs, lens, pinned, arrival_us, digests_host,
                     timeout_us: int = 60_000_000) -> float:
    """Replays requests at the given arrival offsets; returns the worst
    submission delay (us)."""
    ptrs = np.ascontiguousarray(ptrs, dtype=np.uint64)
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
    pin = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.int32)
    late = ctypes.c_double()
    _check(_lib.ht_server_replay(srv, ptrs.ctypes.data, lens.ctypes.data,
                                 None if pin is None else pin.ctypes.data, arr.ctypes.data,
                                 len(lens), _ptr(digests_host), timeout_us, ctypes.byref(late)))
    return late.value


def ht_server_drain(srv: int, timeout_us: int) -> None:
    _check(_lib.ht_server_drain(srv, timeout_us))


def ht_server_stats(srv: int, reset: bool = False) -> dict:
    st = ht_server_stats_t()
    _check(_lib.ht_server_stats(srv, ctypes.byref(st), 1 if reset else 0))
    return st.as_dict()


def ht_server_latencies(srv: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    m = _lib.ht_server_latencies(srv, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
    return out[:m]


def ht_server_destroy(srv: int) -> None:
    _check(_lib.ht_server_destroy(srv))
