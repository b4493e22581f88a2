"""Launch shapes on the GPU: the per-length defaults, the single-string
autotuner over short strings (where 8-execution chunks compete) and the
batch autotuner on the 50,000-string batch.  Every tuned shape must leave
the digests equal to the oracle's, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(built):
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _pair(width, code=None, seed=7):
    from paper_2104_08865_gb300 import Hasher, abi
    code = width if code is None else code
    return Hasher(code, seed_words=abi.ht_seed_expand(seed, code)), abi.ht_seed_expand(seed, code)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_default_shapes_by_length(dev):
    """Strings below 32 MiB default to the block-chunk kernel, longer ones and
    batches to 64-execution warp chunks; the 256-bit-block variant and the
    binary-tree ablation keep 64-execution warp items everywhere; the
    block-chunk kernel is refused for batches."""
    from paper_2104_08865_gb300 import abi
    h, ref = _pair(24)
    for n in (0, 1, 1000, 1 << 20, (32 << 20) - 1):
        assert abi.ht_get_shape(h.ctx, n)["kernel"] == 3, n
    for n in (32 << 20, 1 << 30, 2**64 - 1):
        s = abi.ht_get_shape(h.ctx, n)
        assert s["kernel"] == 1 and s["chunk_levels"] == 2, n
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_set_shape(h.ctx, 2**64 - 1, kernel=3, chunk_levels=2, threads_per_block=256, blocks_per_sm=2)
    assert e.value.code == abi.HT_ERR_ARG
    # the defaults on either side of the boundary, and mid-size strings whose
    # one round is spread over every SM with smaller blocks
    dbuf = inputs.stream_bytes_torch(4, 0, (80 << 20) + 300, dev)
    host = dbuf.cpu().numpy()
    for n in ((32 << 20) - 1, 32 << 20, (40 << 20) + 77, (80 << 20) + 300):
        assert np.array_equal(_u64(h.hash(dbuf, n)), oracle.hash_bytes(24, ref, host[:n])), n
    h.close()
    for code in (24 | abi.HT_BLOCK_256, 24 | abi.HT_TREE_BINARY):
        h, _ = _pair(24, code)
        for n in (1000, 1 << 20, 1 << 30, 2**64 - 1):
            s = abi.ht_get_shape(h.ctx, n)
            assert s["kernel"] == 1 and s["chunk_levels"] == 2
        h.close()


@pytest.mark.parametrize("width", [16, 40])
@pytest.mark.parametrize("n", [64 << 10, (1 << 20) + 77, (6 << 20) + 5])
def test_autotune_short_strings_keeps_digests(dev, width, n):
    """Autotuning a short string's bucket (8-execution chunks among the
    candidates) changes the launch, not the digest."""
    from paper_2104_08865_gb300 import abi
    h, ref = _pair(width)
    best = abi.ht_autotune(h.ctx, n)
    assert abi.ht_get_shape(h.ctx, n) == best
    dbuf = inputs.stream_bytes_torch(5, 0, n, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    assert np.array_equal(_u64(h.hash(dbuf)), want)
    h.close()


def test_autotune_batch_50000_log_uniform(dev):
    """The batch autotuner on the 50,000-string batch (log-uniform 64 B ..
    1 MiB, splitmix64 seed 3, width 24): it stores its pick as the batch
    shape, and the batch's digests under that shape equal the oracle's."""
    from paper_2104_08865_gb300 import abi
    width = 24
    h, ref = _pair(width)
    lens = inputs.log_uniform_lengths(3, 50_000, 64, 1 << 20)
    buf, offs = inputs.packed_batch(3, lens)
    dbuf = torch.from_numpy(buf).to(dev)
    ptrs = torch.tensor([dbuf.data_ptr() + int(o) for o in offs], dtype=torch.int64, device=dev)
    ln = torch.tensor(lens, dtype=torch.int64, device=dev)
    out = torch.zeros((len(lens), 3), dtype=torch.int64, device=dev)
    best = abi.ht_autotune_batch(h.ctx, ptrs, ln, len(lens), out)
    assert abi.ht_get_shape(h.ctx, 2**64 - 1) == best
    want = oracle.hash_many(width, ref, buf, offs, lens)
    assert np.array_equal(_u64(out), want)
    out.zero_()
    abi.ht_hash_batch(h.ctx, ptrs, ln, len(lens), out)
    h.status()
    assert np.array_equal(_u64(out), want)
    h.close()


@pytest.mark.parametrize("shape", [dict(kernel=1, chunk_levels=2, threads_per_block=256, blocks_per_sm=2),
                                   dict(kernel=1, chunk_levels=1, threads_per_block=128, blocks_per_sm=4),
                                   dict(kernel=1, chunk_levels=3, threads_per_block=256, blocks_per_sm=2),
                                   dict(kernel=0, chunk_levels=2, stages=3, threads_per_block=128, blocks_per_sm=2),
                                   dict(kernel=2, chunk_levels=2, threads_per_block=256, blocks_per_sm=2)])
def test_every_batch_family_keeps_digests(dev, shape):
    """Each family the batch autotuner chooses from, set by hand, gives the
    oracle's digests on a mixed batch (short, chunk-sized and multi-chunk
    strings at mixed alignments)."""
    from paper_2104_08865_gb300 import abi
    width = 32
    h, ref = _pair(width)
    abi.ht_set_shape(h.ctx, 2**64 - 1, **shape)
    lens = inputs.log_uniform_lengths(12, 3000, 1, 4 << 20)
    buf, offs = inputs.packed_batch(12, lens)
    offs = [int(o) + (i % 3) for i, o in enumerate(offs)]
    buf = np.concatenate([buf, np.zeros(16, dtype=np.uint8)])
    dbuf = torch.from_numpy(buf).to(dev)
    ptrs = torch.tensor([dbuf.data_ptr() + o for o in offs], dtype=torch.int64, device=dev)
    ln = torch.tensor(lens, dtype=torch.int64, device=dev)
    out = torch.zeros((len(lens), 4), dtype=torch.int64, device=dev)
    abi.ht_hash_batch(h.ctx, ptrs, ln, len(lens), out)
    h.status()
    want = oracle.hash_many(width, ref, buf, offs, lens)
    assert np.array_equal(_u64(out), want)
    h.close()
