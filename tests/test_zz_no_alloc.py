"""The allocation-free entry point, ht_hash_noalloc.

It exists for callers that cannot allocate device memory (inside another
framework's allocator hooks, under another framework's memory pool, or on a
path that cannot take cudaMalloc's synchronisation): it keeps its scratch in a
fixed array the library reserves at load time.  These tests call it through
the C ABI and require the same digests as ht_hash and as the CPU oracle (bit
for bit: the hash is integer arithmetic) on consecutive calls, which share
and re-clear that array.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXEC_BYTES = {16: 1152, 24: 1344, 32: 1344, 40: 960}


@pytest.fixture(scope="module")
def dev(built):
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_noalloc_matches_ht_hash_on_consecutive_calls(dev, width):
    from paper_2104_08865_gb300 import Hasher, abi
    seeds = abi.ht_seed_expand(7, width)
    h = Hasher(width, seed_words=seeds)
    xb = EXEC_BYTES[width]
    # a long string (complete tree groups up to level 4, ragged tail), the
    # same string again, then a short one: each call must clear what the
    # previous one left in the shared array
    long_n = (5 * 512 + 3 * 64 + 2) * 8 * xb + 77
    lens = [long_n, long_n, 9 * 64 * xb + 5, 0]
    data = inputs.stream_bytes_torch(8, 0, long_n + 16, dev)
    host = data.cpu().numpy()
    ref_seeds = oracle.seed_expand(7, oracle.seed_words(width))
    stream = torch.cuda.current_stream()
    for n in lens:
        want = h.hash(data, n)
        got = torch.full((width // 8,), -1, dtype=torch.int64, device=dev)
        abi.ht_hash_noalloc(width, seeds, data.data_ptr(), n, got.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (width, n)
        assert np.array_equal(got.cpu().numpy().view(np.uint64),
                              oracle.hash_bytes(width, ref_seeds, host[:n])), (width, n)
    # a string that does not start on a 16-byte boundary
    n = 70 * xb + 100
    want = h.hash(data, n, offset=3)
    got = torch.empty(width // 8, dtype=torch.int64, device=dev)
    abi.ht_hash_noalloc(width, seeds, data.data_ptr() + 3, n, got.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    assert np.array_equal(got.cpu().numpy().view(np.uint64), oracle.hash_bytes(width, ref_seeds, host[3:3 + n]))
    h.close()


def test_noalloc_rejects_strings_beyond_its_scratch(dev):
    from paper_2104_08865_gb300 import abi
    seeds = abi.ht_seed_expand(7, 40)
    out = torch.empty(5, dtype=torch.int64, device=dev)
    data = torch.empty(16, dtype=torch.uint8, device=dev)
    with pytest.raises(abi.HalftimeError) as e:
        # 12 GB needs more tree groups than the fixed array holds at width 40;
        # the call is refused before any GPU work
        abi.ht_hash_noalloc(40, seeds, data.data_ptr(), 12 * 10**9, out.data_ptr())
    assert e.value.code == abi.HT_ERR_TOO_LONG
    assert "tree groups" in str(e.value)
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_hash_noalloc(40, seeds[:10], data.data_ptr(), 16, out.data_ptr())
    assert e.value.code == abi.HT_ERR_ARG
