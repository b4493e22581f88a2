"""GB300 (sm_103a) HalftimeHash: the CUDA library libhalftime and its binding.

``abi`` mirrors the C ABI of include/halftime.h name for name; ``Hasher`` is
a convenience wrapper over one context that works with torch tensors for
device memory and streams.  All hashing runs in the CUDA kernels.
"""
from __future__ import annotations

import importlib

import numpy as np

__all__ = ["abi", "HalftimeError", "WIDTHS", "Hasher", "Incremental", "Table", "digest_words"]
WIDTHS = (16, 24, 32, 40)


def __getattr__(name):
    # the binding loads libhalftime.so on first use and raises ImportError if
    # the library has not been built (no fallback path exists)
    if name == "abi":
        return importlib.import_module(".abi", __name__)
    if name == "HalftimeError":
        return importlib.import_module(".abi", __name__).HalftimeError
    raise AttributeError(name)


def _abi():
    return importlib.import_module(".abi", __name__)


def digest_words(width: int) -> int:
    """Digest words k of a width code (16/24/32/40, optionally | HT_BLOCK_256)."""
    return (width & 0xFF) // 8


def _device_tensor(t, name: str, dtype=None, min_numel: int = 0):
    """Checks that t is a CUDA tensor (of dtype, with at least min_numel
    elements) before its address reaches a kernel."""
    if not hasattr(t, "is_cuda") or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s, not %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < min_numel:
        raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), min_numel))


class Hasher:
    """One context: a width and an expanded seed on the current device.
    width: 16, 24, 32 or 40, or that value | abi.HT_BLOCK_256 for blocks of
    four words (the 256-bit-block variant)."""

    def __init__(self, width: int, seed64: int = None, seed_words=None, stream=None):
        if seed_words is None:
            seed_words = _abi().ht_seed_expand(seed64 if seed64 is not None else 0, width)
        self.width = width
        self.k = digest_words(width)
        self.seed_words = np.ascontiguousarray(seed_words, dtype=np.uint64)
        self.ctx = _abi().ht_ctx_create(width, self.seed_words, stream)

    def close(self):
        if self.ctx:
            _abi().ht_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # device-resident inputs (torch tensors) --------------------------------
    def hash(self, data, length: int = None, out=None, offset: int = 0, stream=None):
        """Digest of a uint8 CUDA tensor (or a byte range of it) -> int64[k] tensor."""
        import torch
        _device_tensor(data, "data")
        size = data.numel() * data.element_size()
        n = size - offset if length is None else length
        if offset < 0 or n < 0 or offset + n > size:
            raise ValueError("bytes [%d, %d) outside a %d-byte tensor" % (offset, offset + n, size))
        if out is None:
            out = torch.empty(self.k, dtype=torch.int64, device=data.device)
        _device_tensor(out, "out", torch.int64, self.k)
        _abi().ht_hash(self.ctx, data.data_ptr() + offset, n, out.data_ptr(),
                    stream if stream is not None else torch.cuda.current_stream())
        return out

    def hash_batch(self, ptrs_dev, lens_dev, count: int, out=None, stream=None):
        import torch
        _device_tensor(ptrs_dev, "ptrs_dev", torch.int64, count)
        _device_tensor(lens_dev, "lens_dev", torch.int64, count)
        if out is None:
            out = torch.empty((count, self.k), dtype=torch.int64, device=ptrs_dev.device)
        _device_tensor(out, "out", torch.int64, count * self.k)
        _abi().ht_hash_batch(self.ctx, ptrs_dev.data_ptr(), lens_dev.data_ptr(), count,
                          out.data_ptr(), stream if stream is not None else torch.cuda.current_stream())
        return out

    def hash_batch_naive(self, ptrs_host, lens_host, out, stream=None):
        import torch
        ptrs_host = np.ascontiguousarray(ptrs_host, dtype=np.uint64)
        lens_host = np.ascontiguousarray(lens_host, dtype=np.uint64)
        _abi().ht_hash_batch_naive(self.ctx, ptrs_host, lens_host, len(lens_host), out.data_ptr(),
                                stream if stream is not None else torch.cuda.current_stream())
        return out

    def hash_host(self, data_host: np.ndarray, stream=None) -> np.ndarray:
        """Digest of a host buffer (copied in pieces by the library)."""
        import torch
        data_host = np.ascontiguousarray(data_host).view(np.uint8).reshape(-1)
        dig = np.zeros(self.k, dtype=np.uint64)
        _abi().ht_hash_host(self.ctx, data_host.ctypes.data if data_host.size else None,
                         data_host.size, dig.ctypes.data,
                         stream if stream is not None else torch.cuda.current_stream())
        return dig

    def status(self, stream=None):
        _abi().ht_ctx_status(self.ctx, stream)

    def launches(self) -> int:
        return _abi().ht_ctx_launches(self.ctx)

    def incremental(self) -> "Incremental":
        """A handle for one string given in pieces (init / update / final)."""
        return Incremental(self)


class Incremental:
    """Incremental hashing over a Hasher's context: update() with pieces in
    order (CUDA uint8 tensors or host numpy arrays), then final().  The
    digest equals Hasher.hash of the concatenated pieces."""

    def __init__(self, hasher: Hasher):
        self.hasher = hasher
        self.k = hasher.k
        self.h = _abi().ht_inc_create(hasher.ctx)

    def close(self):
        if self.h:
            _abi().ht_inc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream()

    def init(self, stream=None):
        _abi().ht_inc_init(self.h, self._stream(stream))

    def update(self, data, stream=None):
        """Appends a CUDA tensor's bytes (device) or a numpy array's (host)."""
        if isinstance(data, np.ndarray):
            data = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
            _abi().ht_inc_update_host(self.h, data.ctypes.data if data.size else None, data.size,
                                      self._stream(stream))
        else:
            _device_tensor(data, "data")
            n = data.numel() * data.element_size()
            _abi().ht_inc_update(self.h, data.data_ptr() if n else None, n, self._stream(stream))

    def final(self, out=None, stream=None):
        """Digest as a CUDA int64 tensor of k words (uint64 bit patterns)."""
        import torch
        if out is None:
            out = torch.empty(self.k, dtype=torch.int64, device="cuda")
        _abi().ht_inc_final(self.h, out.data_ptr(), self._stream(stream))
        return out

    def status(self, stream=None):
        """Raises if a checked-build launch of this handle skipped an access."""
        _abi().ht_inc_status(self.h, self._stream(stream))

    def length(self) -> int:
        return _abi().ht_inc_length(self.h)

    def granule(self) -> int:
        return _abi().ht_inc_granule(self.h)

    def export_state(self, stream=None) -> bytes:
        return _abi().ht_inc_export(self.h, self._stream(stream))

    def import_state(self, state: bytes, stream=None):
        _abi().ht_inc_import(self.h, state, self._stream(stream))


class Table:
    """Long strings in a device hash table by their digests (ht_table): insert
    digests (a CUDA int64 tensor of shape (count, k), e.g. hash_batch's
    output) to get every entry's representative (the smallest id with an
    equal digest), find digests to get the id of an equal entry."""

    def __init__(self, hasher: Hasher, max_entries: int, seed64: int = 0x7AB1E):
        self.hasher = hasher
        self.k = hasher.k
        self.t = _abi().ht_table_create(hasher.ctx, max_entries, seed64)

    def close(self):
        if self.t:
            _abi().ht_table_destroy(self.t)
            self.t = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream()

    def insert(self, digests, rep: bool = True, stream=None):
        """Inserts the rows of `digests`; returns their representatives (a
        CUDA int32 tensor holding uint32 ids) or None."""
        import torch
        count = digests.shape[0]
        _device_tensor(digests, "digests", torch.int64, count * self.k)
        out = torch.empty(count, dtype=torch.int32, device=digests.device) if rep else None
        _abi().ht_table_insert(self.t, digests, count, out, self._stream(stream))
        return out

    def find(self, digests, stream=None):
        """Ids of entries equal to the rows of `digests` (0xffffffff, i.e. -1
        as int32, where none)."""
        import torch
        count = digests.shape[0]
        _device_tensor(digests, "digests", torch.int64, count * self.k)
        out = torch.empty(count, dtype=torch.int32, device=digests.device)
        _abi().ht_table_find(self.t, digests, count, out, self._stream(stream))
        return out

    def clear(self, stream=None):
        _abi().ht_table_clear(self.t, self._stream(stream))

    def entries(self) -> int:
        return _abi().ht_table_entries(self.t)

    def status(self, stream=None):
        _abi().ht_table_status(self.t, self._stream(stream))
