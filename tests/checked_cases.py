"""Cases run against the checked build (libhalftime_check.so, loaded with
HALFTIME_CHECKED=1 in a process of its own by test_gpu_checked.py): the
range checks must never fire, and every digest must still equal the
oracle's -- single strings, batches (with and without the planner's item
map), incremental pieces and split parts.  Prints "checked: ok" at the end."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2104_08865_gb300 import Hasher, abi, inputs  # noqa: E402

assert abi.CHECKED and abi.ht_build_flags() == abi.HT_BUILD_CHECKED
dev = torch.device("cuda", 0)
torch.cuda.set_device(dev)


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def pair(width, b):
    code = width | (abi.HT_BLOCK_256 if b == 4 else 0)
    ref = oracle.seed_expand(7, oracle.seed_words(width, b))
    return Hasher(code, seed_words=abi.ht_seed_expand(7, code)), ref


# 1. the recorder itself: an index below its limit passes, one above is
#    reported with its value, and reading the status clears it
h, _ = pair(24, 8)
abi.ht_check_probe(h.ctx, 5, 10)
h.status()
abi.ht_check_probe(h.ctx, 12345, 10)
try:
    h.status()
    raise AssertionError("the probe's out-of-range index was not reported")
except abi.HalftimeError as e:
    assert e.code == abi.HT_ERR_DEVICE and "12345" in str(e), e
h.status()
h.close()

# 2. single strings and batches at tree boundaries, both block sizes
for b in (8, 4):
    for width in (16, 24, 32, 40):
        h, ref = pair(width, b)
        xb = oracle.params(width, b)["exec_bytes"]
        Ns = [0, 1, 8, 63, 64, 65, 127, 128, 129, 511, 512, 513, 4096 + 512 + 64 + 9]
        lens = [N * xb + (i * 37) % xb for i, N in enumerate(Ns)] + [5, 700]
        buf, offs = inputs.packed_batch(31, lens)
        want = oracle.hash_many(width, ref, buf, offs, lens, b=b)
        dbuf = torch.from_numpy(buf).to(dev)
        out = torch.empty((len(lens), h.k), dtype=torch.int64, device=dev)
        for i, (o, n) in enumerate(zip(offs, lens)):
            h.hash(dbuf, int(n), out=out[i], offset=int(o))
        h.status()
        assert np.array_equal(u64(out), want), ("single", b, width)
        for sh in (0, 3):
            ptrs = torch.tensor([dbuf.data_ptr() + int(o) + sh for o in offs], dtype=torch.int64, device=dev)
            ln = torch.tensor([max(0, int(n) - sh) for n in lens], dtype=torch.int64, device=dev)
            got = u64(h.hash_batch(ptrs, ln, len(lens)))
            h.status()
            if sh == 0:
                assert np.array_equal(got, want), ("batch", b, width)
            else:
                w2 = np.stack([oracle.hash_bytes(width, ref, buf[int(o) + sh:int(o) + max(sh, int(n))], b=b)
                               for o, n in zip(offs, lens)])
                assert np.array_equal(got, w2), ("unaligned batch", b, width)
        h.close()

# 2a. every kernel family by its launch shape (stream with TMA stages,
#     warp-chunk, hybrid, block-chunk): single strings, aligned and at a
#     3-byte offset, and batches
for width in (24, 40):
    h, ref = pair(width, 8)
    xb = oracle.params(width)["exec_bytes"]
    lens = [0, 7, 5 * xb + 9, 64 * xb, 520 * xb + 3 * xb + 77, 4096 * xb + 1]
    buf, offs = inputs.packed_batch(33, [n + 3 for n in lens])
    dbuf = torch.from_numpy(buf).to(dev)
    for shape in ((0, 2, 3, 128, 1), (1, 2, 3, 256, 2), (2, 2, 3, 256, 2), (3, 2, 3, 256, 2)):
        for bucket in range(64):
            abi.ht_set_shape(h.ctx, 1 << bucket, *shape)
        if shape[0] != 3:
            abi.ht_set_shape(h.ctx, 2**64 - 1, *shape)
        for sh in (0, 3):
            want = np.stack([oracle.hash_bytes(width, ref, buf[int(o) + sh:int(o) + sh + n])
                             for o, n in zip(offs, lens)])
            out = torch.empty((len(lens), h.k), dtype=torch.int64, device=dev)
            for i, (o, n) in enumerate(zip(offs, lens)):
                h.hash(dbuf, n, out=out[i], offset=int(o) + sh)
            h.status()
            assert np.array_equal(u64(out), want), ("family single", width, shape, sh)
            if shape[0] != 3:
                ptrs = torch.tensor([dbuf.data_ptr() + int(o) + sh for o in offs], dtype=torch.int64, device=dev)
                ln = torch.tensor(lens, dtype=torch.int64, device=dev)
                got = u64(h.hash_batch(ptrs, ln, len(lens)))
                h.status()
                assert np.array_equal(got, want), ("family batch", width, shape, sh)
    h.close()

# 2b. a batch of 20,000 strings: the planner's item map and the batch kernel
#     instance that reads it
for b in (8, 4):
    h, ref = pair(24, b)
    rng = np.random.default_rng(b)
    lens = [int(v) for v in rng.integers(0, 3000, 20_000)]
    lens[::1000] = [200_000] * 20  # a few strings of several work items
    buf, offs = inputs.packed_batch(33, lens)
    want = oracle.hash_many(24, ref, buf, offs, lens, b=b)
    dbuf = torch.from_numpy(buf).to(dev)
    ptrs = torch.tensor([dbuf.data_ptr() + int(o) for o in offs], dtype=torch.int64, device=dev)
    ln = torch.tensor(lens, dtype=torch.int64, device=dev)
    before = h.launches()
    got = u64(h.hash_batch(ptrs, ln, len(lens)))
    h.status()
    assert h.launches() - before == 6  # four planner launches, two batch kernels
    assert np.array_equal(got, want), ("item-map batch", b)
    h.close()

# 3. incremental pieces and a string in two parts (512-bit blocks)
for width in (16, 40):
    h, ref = pair(width, 8)
    xb = oracle.params(width)["exec_bytes"]
    # (a piece above 32 MiB takes the warp-chunk update kernel; width 40's
    # updates overlap one another)
    big = (97 << 20) + 5
    n = 600 * 64 * xb + big + 13 * xb + 101
    data = inputs.stream_bytes_torch(32, 0, n, dev)
    want = oracle.hash_bytes(width, ref, data.cpu().numpy())
    if width == 40:
        abi.ht_ctx_set_flags(h.ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
    inc = abi.ht_inc_create(h.ctx)
    cuts = [0, 5, 64 * xb + 3, 300 * 64 * xb + 17, 300 * 64 * xb + 17 + big, n]
    for a, c in zip(cuts[:-1], cuts[1:]):
        abi.ht_inc_update(inc, data.data_ptr() + a, c - a)
    got = torch.empty(h.k, dtype=torch.int64, device=dev)
    abi.ht_inc_final(inc, got.data_ptr())
    abi.ht_inc_status(inc)
    abi.ht_inc_destroy(inc)
    assert np.array_equal(u64(got), want), ("incremental", width)
    parts = [pair(width, 8)[0] for _ in range(2)]
    gran = abi.ht_part_granule(h.ctx)
    cut = 333 * gran
    for p in parts:
        abi.ht_part_begin(p.ctx, n)
    abi.ht_hash_part(parts[0].ctx, data.data_ptr(), 0, cut)
    abi.ht_hash_part(parts[1].ctx, data.data_ptr() + cut, cut, n - cut)
    ptr, words = abi.ht_part_state(parts[1].ctx)
    abi.ht_part_merge(parts[0].ctx, ptr, words)
    abi.ht_finish_parts(parts[0].ctx, got.data_ptr())
    for p in parts:
        p.status()
    assert np.array_equal(u64(got), want), ("parts", width)
    for p in parts:
        p.close()
    h.close()
torch.cuda.synchronize()
print("checked: ok")
