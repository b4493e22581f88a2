"""GPU parity of the binary-tree ablation (width | HT_TREE_BINARY: Badger's
approach, Section 5.2, with Carter and Wegman's tree of Eq. algebraic-badger
consuming all EHC outputs and no final NH): every digest of the CUDA library,
through the C ABI, equals the CPU oracle's bit for bit (integer arithmetic:
the tolerance is zero).

The kernel joins lanes by shuffles, executions in a binary counter per
thread, execution groups by shuffles and work items across warps in pairs,
so the cases put the string's end on every power-of-two boundary of the
execution count up to 2^16, inside and at the end of a 64-execution work
item, and at unaligned addresses.
"""
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
    code = width | abi.HT_TREE_BINARY
    ref = oracle.seed_expand(seed, oracle.seed_words_badger(width))
    lib = abi.ht_seed_expand(seed, code)
    assert np.array_equal(ref, lib)
    return Hasher(code, seed_words=lib), ref


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _batch(h, dbuf, offs, lens):
    ptrs = torch.tensor([dbuf.data_ptr() + int(o) for o in offs], dtype=torch.int64, device=dbuf.device)
    ln = torch.tensor([int(n) for n in lens], dtype=torch.int64, device=dbuf.device)
    out = h.hash_batch(ptrs, ln, len(lens))
    h.status()
    return _u64(out)


def _singles(h, dbuf, offs, lens):
    out = torch.empty((len(lens), h.k), dtype=torch.int64, device=dbuf.device)
    for i, (o, n) in enumerate(zip(offs, lens)):
        h.hash(dbuf, int(n), out=out[i], offset=int(o))
    h.status()
    return _u64(out)


def _boundary_lengths(width):
    xb = oracle.params(width)["exec_bytes"]
    Ns = set()
    for a in range(0, 17):
        for d in (-1, 0, 1):
            if (1 << a) + d >= 0:
                Ns.add((1 << a) + d)
    Ns |= {40, 63, 64 + 37, 3 * 64 + 21, 5 * 64, 7 * 64 + 63, 1000, 4096 + 64 + 8 + 1,
           3 * 4096 + 5 * 64 + 3, 2 * 32768 + 3 * 128 + 64 + 1}
    out = []
    for i, N in enumerate(sorted(Ns)):
        out.append(N * xb)
        out.append(N * xb + (i * 37) % xb)
    return out


SHAPES = {
    "256x2": dict(kernel=1, chunk_levels=2, threads_per_block=256, blocks_per_sm=2),
    "64x1": dict(kernel=1, chunk_levels=2, threads_per_block=64, blocks_per_sm=1),
    "128x32": dict(kernel=1, chunk_levels=2, threads_per_block=128, blocks_per_sm=32),
}


def _set_all(h, shape):
    from paper_2104_08865_gb300 import abi
    for n in [1 << b for b in range(64)] + [2**64 - 1]:
        abi.ht_set_shape(h.ctx, n, **shape)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_binary_tree_boundaries(dev, width, shape):
    """Execution counts around every power of two up to 2^16 with ragged
    tails: one launch per string and one batch launch."""
    h, ref = _pair(width, seed=11)
    _set_all(h, SHAPES[shape])
    lens = _boundary_lengths(width)
    buf, offs = inputs.packed_batch(22, lens)
    want = oracle.hash_many_badger(width, ref, buf, offs, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    got = _singles(h, dbuf, offs, lens)
    bad = np.nonzero(~np.all(got == want, axis=1))[0]
    assert bad.size == 0, "single launches: first mismatches at lengths %s" % [lens[i] for i in bad[:10]]
    got = _batch(h, dbuf, offs, lens)
    bad = np.nonzero(~np.all(got == want, axis=1))[0]
    assert bad.size == 0, "batch: first mismatches at lengths %s" % [lens[i] for i in bad[:10]]
    h.close()


@pytest.mark.parametrize("width", WIDTHS)
def test_binary_all_short_lengths(dev, width):
    """Every length 0..3000 (tail-only strings and up to three executions)
    with random content, in one batch."""
    h, ref = _pair(width)
    lens = list(range(0, 3001))
    buf, offs = inputs.packed_batch(23, lens)
    want = oracle.hash_many_badger(width, ref, buf, offs, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    got = _batch(h, dbuf, offs, lens)
    bad = np.nonzero(~np.all(got == want, axis=1))[0]
    assert bad.size == 0, "first mismatches at lengths %s" % [lens[i] for i in bad[:10]]
    h.close()


@pytest.mark.parametrize("width", WIDTHS)
def test_binary_unaligned_strings(dev, width):
    """Strings starting at every byte offset 1..15 past a 16-byte boundary."""
    h, ref = _pair(width, seed=3)
    xb = oracle.params(width)["exec_bytes"]
    lens = [5, xb - 1, xb + 3, 64 * xb + 11, 96 * xb + 5, 200 * xb + 100]
    src = inputs.stream_bytes(9, 0, max(lens) + 64)
    dbuf = torch.from_numpy(src).to(dev)
    for sh in range(1, 16):
        offs = [sh] * len(lens)
        want = np.stack([oracle.hash_bytes_badger(width, ref, src[sh:sh + n]) for n in lens])
        assert np.array_equal(_singles(h, dbuf, offs, lens), want), sh
        assert np.array_equal(_batch(h, dbuf, offs, lens), want), sh
    h.close()


@pytest.mark.parametrize("width", WIDTHS)
def test_binary_one_gib_string(dev, width):
    """1 GiB of splitmix64(2) bytes, device-resident (the benchmark's input and
    launch configuration for this variant), against the oracle over the whole
    string; the host-input path gives the same digest."""
    h, ref = _pair(width)
    n = 1 << 30
    dbuf = inputs.stream_bytes_torch(2, 0, n, dev)
    got = _u64(h.hash(dbuf))
    h.status()
    host = dbuf.cpu().numpy()
    want = oracle.hash_bytes_badger(width, ref, host)
    assert np.array_equal(got, want)
    pinned = torch.empty(n, dtype=torch.uint8).pin_memory()
    pinned.copy_(torch.from_numpy(host))
    assert np.array_equal(h.hash_host(pinned.numpy()), want)
    h.close()


def test_binary_batch_log_uniform(dev):
    """20,000 strings, lengths log-uniform in [64 B, 1 MiB] (splitmix64 seed
    3), width 24: the batch launch, one launch per string and the oracle
    agree on every digest."""
    width = 24
    h, ref = _pair(width)
    lens = inputs.log_uniform_lengths(3, 20_000, 64, 1 << 20)
    buf, offs = inputs.packed_batch(3, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    got = _batch(h, dbuf, offs, lens)
    naive = torch.empty((len(lens), 3), dtype=torch.int64, device=dev)
    h.hash_batch_naive([dbuf.data_ptr() + int(o) for o in offs], lens, naive)
    assert np.array_equal(_u64(naive), got)
    want = oracle.hash_many_badger(width, ref, buf, offs, lens)
    assert np.array_equal(got, want)
    h.close()


def test_binary_shape_rules_and_refusals(dev):
    """The autotuner considers the warp-chunk kernel with 64-execution items
    only; other shapes are refused; incremental handles, parts and the
    allocation-free call refuse the ablation."""
    from paper_2104_08865_gb300 import abi
    width = 32
    h, ref = _pair(width)
    n = 48 << 20
    dbuf = inputs.stream_bytes_torch(6, 0, n, dev)
    before = _u64(h.hash(dbuf))
    best = abi.ht_autotune(h.ctx, n)
    assert best["kernel"] == 1 and best["chunk_levels"] == 2
    assert np.array_equal(_u64(h.hash(dbuf)), before)
    assert np.array_equal(before, oracle.hash_bytes_badger(width, ref, dbuf.cpu().numpy()))
    for bad in (dict(kernel=0, stages=3, threads_per_block=192, blocks_per_sm=1),
                dict(kernel=2, threads_per_block=256, blocks_per_sm=2),
                dict(kernel=1, chunk_levels=3, threads_per_block=256, blocks_per_sm=2),
                dict(kernel=1, chunk_levels=1, threads_per_block=256, blocks_per_sm=2)):
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_set_shape(h.ctx, n, **bad)
        assert e.value.code == abi.HT_ERR_ARG
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_inc_create(h.ctx)
    assert e.value.code == abi.HT_ERR_WIDTH
    assert abi.ht_part_granule(h.ctx) == 0
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_part_begin(h.ctx, 1 << 20)
    assert e.value.code == abi.HT_ERR_WIDTH
    out = torch.empty(4, dtype=torch.int64, device=dev)
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_hash_noalloc(width | abi.HT_TREE_BINARY, ref, dbuf.data_ptr(), 1000, out.data_ptr())
    assert e.value.code == abi.HT_ERR_WIDTH
    h.close()


def test_binary_serving_alone_vs_mix(dev):
    """A server over a context of the ablation: requests of mixed sizes,
    device-resident, every digest equal to the one hashed alone and to the
    oracle's on a sample."""
    from paper_2104_08865_gb300 import abi
    width = 40
    h, ref = _pair(width)
    rng = np.random.default_rng(31)
    n = 120
    pool = 64 << 20
    pool_dev = inputs.stream_bytes_torch(8, 0, pool, dev)
    lens = inputs.log_uniform_lengths(17, n, 256, 4 << 20)
    offs = rng.integers(0, pool - (4 << 20), n)
    ptrs = pool_dev.data_ptr() + offs
    arrivals = np.sort(rng.uniform(0, 10_000, n))
    srv = abi.ht_server_create(h.ctx, 128 << 20, n_streams=2, max_batch=16)
    try:
        dig = np.zeros((n, 5), dtype=np.uint64)
        abi.ht_server_replay(srv, ptrs, lens, np.zeros(n, dtype=np.int32), arrivals, dig)
        assert abi.ht_server_stats(srv)["completed"] == n
    finally:
        abi.ht_server_destroy(srv)
    alone = torch.empty((n, 5), dtype=torch.int64, device=dev)
    for i in range(n):
        h.hash(pool_dev, int(lens[i]), out=alone[i], offset=int(offs[i]))
    assert np.array_equal(dig, _u64(alone))
    host = pool_dev.cpu().numpy()
    for i in range(0, n, 10):
        o, ln = int(offs[i]), int(lens[i])
        assert np.array_equal(dig[i], oracle.hash_bytes_badger(width, ref, host[o:o + ln]))
    h.close()
