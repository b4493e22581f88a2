"""Batches holding multi-gigabyte strings beside small ones: every string's
tree-group slots come from the device planner, so strings of 8^7 and more
executions test its per-string offsets at high levels, with the
aligned-only batch kernel and (one string at an odd address) the general
one; every digest bit-exact against the oracle (width 40, both block
sizes)."""
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


@pytest.mark.parametrize("b", [8, 4])
def test_batch_with_gigabyte_strings(dev, b):
    from paper_2104_08865_gb300 import Hasher, abi
    width = 40
    code = width | (abi.HT_BLOCK_256 if b == 4 else 0)
    xb = oracle.params(width, b)["exec_bytes"]
    rng = np.random.default_rng(b)
    big = [(8**7 + 3 * 8**6 + 2 * 8**3 + 5) * xb + 101, (8**7 + 8**4 + 1) * xb + 7]
    small = [int(v) for v in rng.integers(0, 100_000, 30)]
    lens = big + small
    total = sum(lens) + 64 * len(lens) + 4096
    free, _ = torch.cuda.mem_get_info()
    if free < total + (4 << 30):
        pytest.skip("needs %.1f GB of free device memory" % ((total + (4 << 30)) / 1e9))
    data = inputs.stream_bytes_torch(43, 0, total, dev)
    host = data.cpu().numpy()
    ref = oracle.seed_expand(7, oracle.seed_words(width, b))
    want = {}
    h = Hasher(code, seed_words=abi.ht_seed_expand(7, code))
    for shift in (0, 3):
        # shift 0: every string 256-byte aligned (the aligned-only kernel);
        # shift 3: the second big string starts 3 bytes past a boundary (the
        # general kernel takes the batch)
        offs, o = [], 0
        for i, n in enumerate(lens):
            offs.append(o + (shift if i == 1 else 0))
            o = (offs[-1] + n + 255) // 256 * 256
        assert o <= total
        ptrs = torch.tensor([data.data_ptr() + x for x in offs], dtype=torch.int64, device=dev)
        ln = torch.tensor(lens, dtype=torch.int64, device=dev)
        got = h.hash_batch(ptrs, ln, len(lens)).cpu().numpy().view(np.uint64)
        h.status()
        for i, (x, n) in enumerate(zip(offs, lens)):
            if (x, n) not in want:
                want[x, n] = oracle.hash_bytes(width, ref, host[x:x + n], b=b)
            assert np.array_equal(got[i], want[x, n]), (shift, i, n)
    h.close()
