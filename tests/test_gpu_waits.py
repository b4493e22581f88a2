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
