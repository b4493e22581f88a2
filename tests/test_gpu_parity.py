"""GPU parity: every digest of the CUDA library, through the C ABI, equals the
CPU oracle's bit for bit (integer arithmetic: the tolerance is zero).

Inputs come from the seeded generators of paper_2104_08865_gb300.inputs; the
oracle's seeds come from the oracle's own splitmix64, the library's from
ht_seed_expand.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIDTHS = (16, 24, 32, 40)


@pytest.fixture(scope="module")
def dev(built):
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _pair(width, seed=7):
    from paper_2104_08865_gb300 import Hasher, abi
    ref = oracle.seed_expand(seed, oracle.seed_words(width))
    lib = abi.ht_seed_expand(seed, width)
    return Hasher(width, seed_words=lib), ref


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _batch(h, dbuf, offs, lens, base_off=0):
    ptrs = torch.tensor([dbuf.data_ptr() + base_off + int(o) for o in offs], dtype=torch.int64,
                        device=dbuf.device)
    ln = torch.tensor([int(n) for n in lens], dtype=torch.int64, device=dbuf.device)
    out = h.hash_batch(ptrs, ln, len(lens))
    h.status()
    return _u64(out)


def _singles(h, dbuf, offs, lens, base_off=0):
    out = torch.empty((len(lens), h.k), dtype=torch.int64, device=dbuf.device)
    for i, (o, n) in enumerate(zip(offs, lens)):
        h.hash(dbuf, int(n), out=out[i], offset=base_off + int(o))
    return _u64(out)


def test_c1_hh16_1000_strings_of_4096(dev):
    """1,000 strings of 4,096 random bytes (splitmix64 seed 1), HH16, seed 7."""
    h, ref = _pair(16)
    lens = [4096] * 1000
    buf, offs = inputs.packed_batch(1, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    want = oracle.hash_many(16, ref, buf, offs, lens)
    assert np.array_equal(_batch(h, dbuf, offs, lens), want)
    assert np.array_equal(_singles(h, dbuf, offs, lens), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_edge_sweep_all_lengths_and_contents(dev, width):
    """Every length 0..8192 with zero, 0xFF, 8-byte-pattern and random content."""
    h, ref = _pair(width)
    lens, parts = [], []
    for kind in ("zero", "ff", "pattern8", "random"):
        for n in range(0, 8193):
            lens.append(n)
            parts.append(inputs.pattern_bytes(kind, n))
    slots = [(n + 255) // 256 * 256 for n in lens]
    offs = np.concatenate([[0], np.cumsum(slots)[:-1]]).astype(np.int64)
    buf = np.zeros(int(sum(slots)) + 256, dtype=np.uint8)
    for o, p in zip(offs, parts):
        buf[o:o + len(p)] = p
    want = oracle.hash_many(width, ref, buf, offs, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    got = _batch(h, dbuf, offs, lens)
    bad = np.nonzero(~np.all(got == want, axis=1))[0]
    assert bad.size == 0, "first mismatches at lengths %s" % [lens[i] for i in bad[:10]]
    sel = list(range(0, len(lens), 61))
    got1 = _singles(h, dbuf, offs[sel], [lens[i] for i in sel])
    assert np.array_equal(got1, want[sel])


def _boundary_lengths(width):
    xb = oracle.params(width)["exec_bytes"]
    Ns = [1, 7, 8, 9, 63, 64, 65, 71, 72, 511, 512, 513, 575, 4095, 4096, 4097, 4096 + 512 + 64 + 9,
          32767, 32768, 32769, 8 * 4096 + 3 * 512 + 5 * 64 + 7]
    out = []
    for i, N in enumerate(Ns):
        out.append(N * xb)
        out.append(N * xb + (i * 37) % xb)
    return out


SHAPES = {
    "stream-r2-w8": dict(kernel=0, stages=2, threads_per_block=256, blocks_per_sm=1),
    "stream-r3-w6": dict(kernel=0, stages=3, threads_per_block=192, blocks_per_sm=1),
    "stream-r4-w2x2": dict(kernel=0, stages=4, threads_per_block=64, blocks_per_sm=2),
    "range-256x2": dict(kernel=2, threads_per_block=256, blocks_per_sm=2),
    "range-64x1": dict(kernel=2, threads_per_block=64, blocks_per_sm=1),
    "chunk-L1": dict(kernel=1, chunk_levels=1, threads_per_block=256, blocks_per_sm=32),
    "chunk-L2": dict(kernel=1, chunk_levels=2, threads_per_block=256, blocks_per_sm=32),
    "chunk-L3": dict(kernel=1, chunk_levels=3, threads_per_block=128, blocks_per_sm=32),
    "block-256x2": dict(kernel=3, threads_per_block=256, blocks_per_sm=2),
    "block-256x8": dict(kernel=3, threads_per_block=256, blocks_per_sm=8),
}


def _set_all(h, shape):
    """Every length bucket, and the batch shape unless the kernel serves
    single strings only (the block-chunk kernel)."""
    from paper_2104_08865_gb300 import abi
    for n in [1 << b for b in range(64)] + ([2**64 - 1] if shape["kernel"] < 3 else []):
        abi.ht_set_shape(h.ctx, n, **shape)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_chunk_and_tree_boundaries(dev, width, shape):
    """Execution counts around every f^l boundary (partial stages and chunks,
    pending roots at each level, complete upper groups) with ragged tails,
    for both kernel families and several launch shapes."""
    h, ref = _pair(width, seed=11)
    _set_all(h, SHAPES[shape])
    lens = _boundary_lengths(width)
    buf, offs = inputs.packed_batch(21, lens)
    want = oracle.hash_many(width, ref, buf, offs, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    assert np.array_equal(_singles(h, dbuf, offs, lens), want)
    assert np.array_equal(_batch(h, dbuf, offs, lens), want)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("shape", ["stream-r3-w6", "chunk-L2", "range-256x2", "block-256x2"])
def test_unaligned_strings(dev, width, shape):
    """Strings starting at every byte offset 1..15 past a 16-byte boundary."""
    h, ref = _pair(width, seed=3)
    _set_all(h, SHAPES[shape])
    xb = oracle.params(width)["exec_bytes"]
    lens = [5, xb - 1, xb + 3, 64 * xb + 11, 70 * xb + 100]
    src = inputs.stream_bytes(9, 0, max(lens) + 64)
    dbuf = torch.from_numpy(src).to(dev)
    for sh in range(1, 16):
        offs = [sh] * len(lens)
        want = np.stack([oracle.hash_bytes(width, ref, src[sh:sh + n]) for n in lens])
        assert np.array_equal(_singles(h, dbuf, offs, lens), want), sh
        assert np.array_equal(_batch(h, dbuf, offs, lens), want), sh


@pytest.mark.parametrize("width", WIDTHS)
def test_c2_one_gib_string(dev, width):
    """1 GiB of splitmix64(2) bytes, device-resident (the benchmark's input and
    launch configuration), bit-exact against the oracle over the whole string;
    the host-input path gives the same digest."""
    h, ref = _pair(width)
    n = 1 << 30
    dbuf = inputs.stream_bytes_torch(2, 0, n, dev)
    got = _u64(h.hash(dbuf))
    host = dbuf.cpu().numpy()
    want = oracle.hash_bytes(width, ref, host)
    assert np.array_equal(got, want)
    for name in ("chunk-L2", "stream-r3-w6", "block-256x2"):
        _set_all(h, SHAPES[name])
        assert np.array_equal(_u64(h.hash(dbuf)), want), name
    pinned = torch.empty(n, dtype=torch.uint8).pin_memory()
    pinned.copy_(torch.from_numpy(host))
    assert np.array_equal(h.hash_host(pinned.numpy()), want)


@pytest.mark.parametrize("shape", ["stream-r3-w6", "chunk-L2", "range-256x2"])
def test_c4_batch_50000_log_uniform(dev, shape):
    """50,000 strings, lengths log-uniform in [64 B, 1 MiB] (splitmix64 seed 3),
    HH24: the batch launch, one launch per string and the oracle agree on
    every digest."""
    width = 24
    h, ref = _pair(width)
    _set_all(h, SHAPES[shape])
    lens = inputs.log_uniform_lengths(3, 50_000, 64, 1 << 20)
    buf, offs = inputs.packed_batch(3, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    got = _batch(h, dbuf, offs, lens)
    naive = torch.empty((len(lens), 3), dtype=torch.int64, device=dev)
    h.hash_batch_naive([dbuf.data_ptr() + int(o) for o in offs], lens, naive)
    assert np.array_equal(_u64(naive), got)
    want = oracle.hash_many(width, ref, buf, offs, lens)
    assert np.array_equal(got, want)


def test_batch_of_a_million_short_strings(dev):
    """1,050,000 strings of 0 .. 1400 bytes (tail-only, or one execution and
    a tail), width 16: 1026 planner tiles, more than the 1024 that one pass
    of the totals kernel scans; every digest against the oracle."""
    from paper_2104_08865_gb300 import abi
    width = 16
    h, ref = _pair(width)
    rng = np.random.default_rng(77)
    lens = rng.integers(0, 1401, size=1_050_000).astype(np.int64)
    buf, offs = inputs.packed_batch(5, lens)
    abi.ht_ctx_reserve(h.ctx, int(buf.size), len(lens))
    dbuf = torch.from_numpy(buf).to(dev)
    got = _batch(h, dbuf, offs, lens)
    h.status()
    assert np.array_equal(got, oracle.hash_many(width, ref, buf, offs, lens))


@pytest.mark.parametrize("width", [24, 40])
def test_autotuned_shape_keeps_digests(dev, width):
    from paper_2104_08865_gb300 import abi
    h, ref = _pair(width)
    n = 48 << 20
    best = abi.ht_autotune(h.ctx, n)
    assert best["kernel"] in (0, 1, 2, 3)
    assert abi.ht_get_shape(h.ctx, n) == best
    dbuf = inputs.stream_bytes_torch(5, 0, n + 333, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    assert np.array_equal(_u64(h.hash(dbuf)), want)


def test_launch_counter_counts_kernels(dev):
    h, _ = _pair(32)
    dbuf = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
    before = h.launches()
    h.hash(dbuf)
    ptrs = torch.tensor([dbuf.data_ptr()] * 3, dtype=torch.int64, device=dev)
    ln = torch.tensor([10, 1000, 100000], dtype=torch.int64, device=dev)
    h.hash_batch(ptrs, ln, 3)
    torch.cuda.synchronize()
    from paper_2104_08865_gb300 import abi
    batch_kernel = abi.ht_get_shape(h.ctx, 2**64 - 1)["kernel"]
    # one hash kernel, then the planner (one launch for batches of up to
    # 1024 strings) and the batch kernels (an aligned and a general one,
    # except for the stream family)
    assert h.launches() - before == 1 + {0: 2, 1: 3, 2: 3}[batch_kernel]
    if batch_kernel == 1:
        # more than 1024 strings: the multi-block planner (three launches);
        # 16,384 or more: a fourth planner launch writes the item -> string map
        for n, launches in ((2_000, 5), (20_000, 6)):
            ptrs = torch.full((n,), dbuf.data_ptr(), dtype=torch.int64, device=dev)
            ln = torch.full((n,), 100, dtype=torch.int64, device=dev)
            before = h.launches()
            h.hash_batch(ptrs, ln, n)
            torch.cuda.synchronize()
            assert h.launches() - before == launches, n


def test_python_layer_rejects_bad_tensors(dev):
    """The convenience layer checks tensors before their addresses reach a
    kernel: host tensors, wrong dtypes and ranges past the end are refused."""
    from paper_2104_08865_gb300 import Table
    h, _ = _pair(16)
    d = torch.zeros(1000, dtype=torch.uint8, device=dev)
    with pytest.raises(ValueError):
        h.hash(torch.zeros(1000, dtype=torch.uint8))  # host tensor
    with pytest.raises(ValueError):
        h.hash(d, length=1001)
    with pytest.raises(ValueError):
        h.hash(d, length=10, offset=995)
    ptrs = torch.tensor([d.data_ptr()], dtype=torch.int64, device=dev)
    with pytest.raises(ValueError):
        h.hash_batch(ptrs, torch.tensor([10], dtype=torch.int32, device=dev), 1)
    with pytest.raises(ValueError):
        h.hash_batch(ptrs, torch.tensor([10], dtype=torch.int64, device=dev), 2)
    with h.incremental() as inc:
        with pytest.raises(ValueError):
            inc.update(torch.zeros(10, dtype=torch.uint8))
    with Table(h, max_entries=4) as t:
        with pytest.raises(ValueError):
            t.insert(torch.zeros((2, 2), dtype=torch.int64))
    # the valid forms still work
    assert h.hash(d, length=10, offset=990).shape == (2,)


@pytest.mark.parametrize("width", WIDTHS)
def test_rekey_matches_fresh_context(dev, width):
    from paper_2104_08865_gb300 import abi
    h, _ = _pair(width, seed=1)
    ref2 = oracle.seed_expand(99, oracle.seed_words(width))
    abi.ht_ctx_rekey(h.ctx, abi.ht_seed_expand(99, width))
    data = inputs.stream_bytes(6, 0, 3 * 64 * oracle.params(width)["exec_bytes"] + 5)
    got = _u64(h.hash(torch.from_numpy(data).to(dev)))
    assert np.array_equal(got, oracle.hash_bytes(width, ref2, data))


@pytest.mark.parametrize("shape", [None, "block-256x2"])
def test_overlapped_launches_keep_digests(dev, shape):
    """Back-to-back hashes with HT_FLAG_OVERLAP_LAUNCHES (each launch may
    start while the previous one drains) on two contexts sharing one stream,
    over sizes from empty to several rounds of chunks, with the default
    shapes and with the block-chunk kernel for every length: every digest
    equals the oracle's."""
    from paper_2104_08865_gb300 import abi
    pairs = [_pair(24, seed=3), _pair(40, seed=4)]
    for h, _ in pairs:
        abi.ht_ctx_set_flags(h.ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
        if shape:
            _set_all(h, SHAPES[shape])
    lens = [0, 17, 5000, 300_000, 9 << 20, (1 << 26) + 12345, 3 << 20, 1 << 27]
    data = inputs.stream_bytes_torch(15, 0, max(lens), dev)
    outs = []
    for rep in range(2):
        for n in lens:
            for h, _ in pairs:
                outs.append((h, n, h.hash(data, n)))  # no synchronisation in between
    torch.cuda.synchronize()
    host = data.cpu().numpy()
    want = {}
    for h, ref in pairs:
        for n in lens:
            want[(h.width, n)] = oracle.hash_bytes(h.width, ref, host[:n])
    for h, n, got in outs:
        assert np.array_equal(_u64(got), want[(h.width, n)]), (h.width, n)


def test_default_launches_hash_the_previous_digest(dev):
    """Without the overlap flag a call may hash what the previous call wrote:
    the digest of a string, hashed again, equals the oracle's chain."""
    h, ref = _pair(32)
    data = inputs.stream_bytes_torch(16, 0, 50 << 20, dev)
    d1 = h.hash(data)
    d2 = h.hash(d1.view(torch.uint8))
    want1 = oracle.hash_bytes(32, ref, data.cpu().numpy())
    want2 = oracle.hash_bytes(32, ref, want1.view(np.uint8))
    assert np.array_equal(_u64(d1), want1)
    assert np.array_equal(_u64(d2), want2)


@pytest.mark.parametrize("pinned_mode", [0, 1])
def test_serving_alone_vs_mix(dev, pinned_mode):
    """Requests of mixed sizes (device-resident and pinned host, the latter
    read in place by the kernel or staged through device memory) arrive while
    others are on the GPU; every digest equals the one hashed alone, and the
    oracle's on a sample."""
    from paper_2104_08865_gb300 import abi
    width = 32
    h, ref = _pair(width)
    rng = np.random.default_rng(12)
    n = 240
    pool = 96 << 20
    pool_dev = inputs.stream_bytes_torch(7, 0, pool, dev)
    pool_host = torch.empty(pool, dtype=torch.uint8).pin_memory()
    pool_host.copy_(pool_dev)
    torch.cuda.synchronize()
    lens = inputs.log_uniform_lengths(13, n, 256, 4 << 20)
    offs = rng.integers(0, pool - (4 << 20), n)  # any alignment
    pinned = rng.integers(0, 2, n).astype(np.int32)
    ptrs = np.where(pinned == 1, pool_host.data_ptr() + offs, pool_dev.data_ptr() + offs)
    arrivals = np.sort(rng.uniform(0, 20_000, n))
    srv = abi.ht_server_create(h.ctx, 256 << 20, n_streams=3, max_batch=32, pinned_mode=pinned_mode)
    try:
        dig = np.zeros((n, 4), dtype=np.uint64)
        abi.ht_server_replay(srv, ptrs, lens, pinned, arrivals, dig)
        st = abi.ht_server_stats(srv)
        assert st["completed"] == n and st["batches"] > 1
    finally:
        abi.ht_server_destroy(srv)
    alone = torch.empty((n, 4), dtype=torch.int64, device=dev)
    for i in range(n):
        h.hash(pool_dev, int(lens[i]), out=alone[i], offset=int(offs[i]))
    assert np.array_equal(dig, _u64(alone))
    host = pool_dev.cpu().numpy()
    for i in range(0, n, 12):
        o, ln = int(offs[i]), int(lens[i])
        assert np.array_equal(dig[i], oracle.hash_bytes(width, ref, host[o:o + ln]))


@pytest.mark.parametrize("width", WIDTHS)
def test_c3_collision_sweep(dev, width):
    """100,000 pairs of 64 KiB random strings (splitmix64 seed 4) that differ
    in one 32-bit word, hashed under 1,000 seeds (splitmix64 seed 11 outputs):
    no full-width collision among the 10^8 pairs (the bound of Section 6.2,
    2^-32k (2^kp + h^k + 1), predicts about 1e-10 of them), and a 10^4-hash
    sample agrees with the oracle bit for bit.
    A diagnostic that can fail: for the pairs whose changed word lies in the
    tail, the outputs differ by the difference of one NH term, (A)(B) -
    (A')(B) or (A)(B) - (A)(B'), with the unchanged factor uniform over the
    seeds; so the low 16 bits of each output word collide with probability
    exactly 2^(min(v, 16) - 16), v the lowest set bit of the word's XOR
    difference.  The count over all seeds must lie within six standard
    deviations of the sum of those probabilities, for every output word.
    (For changes in the EHC input no such exact rate exists: there the
    difference passes through further multiplications.)"""
    from paper_2104_08865_gb300 import abi
    pairs, n, seeds = 100_000, 1 << 16, 1000
    rng = np.random.default_rng(width)
    both = torch.empty((2, pairs, n), dtype=torch.uint8, device=dev)
    both[0].copy_(inputs.stream_bytes_torch(4, 0, pairs * n, dev).view(pairs, n))
    both[1].copy_(both[0])
    base, flipped = both[0], both[1]
    words = flipped.view(torch.int32)
    pos_np = rng.integers(0, n // 4, pairs)
    flip_np = rng.integers(1, 2**32, pairs, dtype=np.uint64)
    pos = torch.from_numpy(pos_np).to(dev)
    flip = torch.from_numpy(flip_np.astype(np.uint32).view(np.int32)).to(dev)
    rows = torch.arange(pairs, device=dev)
    words[rows, pos] ^= flip
    ptrs = both.data_ptr() + torch.arange(2 * pairs, device=dev, dtype=torch.int64) * n
    lens = torch.full((2 * pairs,), n, dtype=torch.int64, device=dev)
    seed64 = inputs.splitmix64_words(11, 0, seeds)
    h, _ = _pair(width)
    abi.ht_ctx_reserve(h.ctx, 2 * pairs * n, 2 * pairs)
    k = width // 8
    # pairs whose changed 32-bit word lies in the tail, and their rates
    tail_start = (n // oracle.params(width)["exec_bytes"]) * oracle.params(width)["exec_bytes"]
    in_tail = 4 * pos_np >= tail_start
    v = np.array([min((int(f) & -int(f)).bit_length() - 1, 16) for f in flip_np])
    p = np.where(in_tail, 2.0 ** (v - 16), 0.0)
    tail_rows = torch.from_numpy(np.nonzero(in_tail)[0]).to(dev)
    out = torch.empty((2 * pairs, k), dtype=torch.int64, device=dev)
    full = 0
    window = torch.zeros(k, dtype=torch.int64, device=dev)
    for i in range(seeds):
        abi.ht_ctx_rekey(h.ctx, abi.ht_seed_expand(int(seed64[i]), width))
        abi.ht_hash_batch(h.ctx, ptrs, lens, 2 * pairs, out)
        a, b = out[:pairs], out[pairs:]
        full += int(torch.all(a == b, dim=1).sum())
        window += (((a[tail_rows] ^ b[tail_rows]) & 0xFFFF) == 0).sum(dim=0)
        if i == 0:
            sample = _u64(torch.cat([a[:5000], b[:5000]]))
    h.status()
    assert full == 0
    mean = seeds * p.sum()
    sd = math.sqrt(seeds * (p * (1 - p)).sum())
    assert in_tail.sum() > 100 and mean > 20
    for t, c in enumerate(window.cpu().tolist()):
        assert abs(c - mean) <= 6 * sd + 1, (t, c, mean, sd)
    ref = oracle.seed_expand(int(seed64[0]), oracle.seed_words(width))
    host = torch.cat([base[:5000], flipped[:5000]]).cpu().numpy().reshape(-1)
    offs = np.arange(10_000, dtype=np.int64) * n
    want = oracle.hash_many(width, ref, host, offs, [n] * 10_000)
    assert np.array_equal(sample, want)


@pytest.mark.parametrize("width", WIDTHS)
def test_block_chunk_kernel_interleaved(dev, width):
    """Strings of 0 to 520 whole 64-execution chunks hashed by the block-chunk
    kernel (the default below 32 MiB), around each 8^l boundary of the
    chunk count and with partial chunks and tails, one after another on one
    context, then again in reverse order: a launch that leaves anything in
    the scratch spoils the next one."""
    h, ref = _pair(width, seed=19)
    xb = oracle.params(width)["exec_bytes"]
    lens = []
    for i, c in enumerate([0, 1, 2, 7, 8, 9, 63, 64, 65, 100, 511, 512, 513, 520]):
        for r in (0, 5, 63):
            if c * 64 + r:
                lens.append((c * 64 + r) * xb + (i * 41 + r) % xb)
    buf, offs = inputs.packed_batch(31, lens)
    want = oracle.hash_many(width, ref, buf, offs, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    for rep in range(2):
        order = list(range(len(lens))) if rep == 0 else list(range(len(lens)))[::-1]
        out = torch.empty((len(lens), h.k), dtype=torch.int64, device=dev)
        for i in order:
            h.hash(dbuf, int(lens[i]), out=out[i], offset=int(offs[i]))
        h.status()
        got = _u64(out)
        bad = np.nonzero(~np.all(got == want, axis=1))[0]
        assert bad.size == 0, (rep, [lens[i] // xb for i in bad[:10]])
