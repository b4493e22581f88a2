"""Failure detection on the GPU without a fault: a bounded device wait (the
stream kernel's wait on a shared-memory stage) is made to run out on a
stage that nothing fills; the kernel reports it in the status word and
returns, the host reads HT_ERR_DEVICE, and the context keeps hashing
correctly."""
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


def test_bounded_wait_runs_out_and_is_reported(dev):
    from paper_2104_08865_gb300 import Hasher, abi
    width = 24
    ref = oracle.seed_expand(7, oracle.seed_words(width))
    h = Hasher(width, seed_words=abi.ht_seed_expand(7, width))
    for cycles in (1, 2_000_000):  # at once, and after about a millisecond
        abi.ht_wait_probe(h.ctx, cycles)
        with pytest.raises(abi.HalftimeError) as e:
            h.status()
        assert e.value.code == abi.HT_ERR_DEVICE and "gave up waiting" in str(e.value)
        h.status()  # reading the status cleared it
    # the context is still usable, with every kernel family
    n = 70 * 1344 * 64 + 333
    data = inputs.stream_bytes_torch(44, 0, n, dev)
    want = oracle.hash_bytes(width, ref, data.cpu().numpy())
    for shape in (dict(kernel=1, chunk_levels=2, threads_per_block=256, blocks_per_sm=2),
                  dict(kernel=0, stages=3, threads_per_block=192, blocks_per_sm=1)):
        abi.ht_set_shape(h.ctx, n, **shape)
        got = h.hash(data).cpu().numpy().view(np.uint64)
        h.status()
        assert np.array_equal(got, want), shape
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_wait_probe(h.ctx, 0)
    assert e.value.code == abi.HT_ERR_ARG
    h.close()


def test_stage_wait_runs_out_in_a_hash_and_the_context_recovers(dev):
    """The stream kernel itself, hashing, with a stage-wait limit of a few
    cycles: its first stage wait runs out while the copy is in flight (the
    wait that lets issued copies land keeps its normal limit, so nothing is
    left in flight); the status reads HT_ERR_DEVICE, reading it clears the
    tree groups and string sums that the abandoned work left, and the next
    hashes on the same context (both families) equal the oracle's."""
    from paper_2104_08865_gb300 import Hasher, abi
    width = 32
    ref = oracle.seed_expand(5, oracle.seed_words(width))
    h = Hasher(width, seed_words=abi.ht_seed_expand(5, width))
    n = 300 * 1344 * 64 + 71  # tree groups up to level 4 half built when warps give up
    data = inputs.stream_bytes_torch(45, 0, n, dev)
    want = oracle.hash_bytes(width, ref, data.cpu().numpy())
    stream_shape = dict(kernel=0, stages=3, threads_per_block=192, blocks_per_sm=1)
    abi.ht_set_shape(h.ctx, n, **stream_shape)
    abi.ht_testing_set_wait_cycles(h.ctx, 2)
    h.hash(data)
    with pytest.raises(abi.HalftimeError) as e:
        h.status()
    assert e.value.code == abi.HT_ERR_DEVICE and "gave up waiting" in str(e.value)
    abi.ht_testing_set_wait_cycles(h.ctx, 0)
    for shape in (stream_shape, dict(kernel=1, chunk_levels=2, threads_per_block=256, blocks_per_sm=2)):
        abi.ht_set_shape(h.ctx, n, **shape)
        got = h.hash(data).cpu().numpy().view(np.uint64)
        h.status()
        assert np.array_equal(got, want), shape
    h.close()
