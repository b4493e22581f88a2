"""Deep trees: strings of more than 8^8 executions, so that tree groups
complete up to level 7 and the scratch slots of every level up to 8 are
used, bit-exact against the oracle over the whole string (width 40, the
smallest execution: 960 bytes with 512-bit blocks, 480 with 256-bit
blocks).  The other parity tests stop at about 8^6 executions."""
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
def test_string_beyond_eight_levels(dev, b):
    from paper_2104_08865_gb300 import Hasher, abi
    width = 40
    code = width | (abi.HT_BLOCK_256 if b == 4 else 0)
    xb = oracle.params(width, b)["exec_bytes"]
    # base-8 digits of N: 1 at level 8, 1 at level 7, 5 at level 4, 3 at
    # level 0 -- complete groups up to level 7, pending roots at four levels
    N = 8**8 + 8**7 + 5 * 8**4 + 3
    n = N * xb + xb // 2 + 37  # a ragged tail, shorter than one execution
    free, _ = torch.cuda.mem_get_info()
    if free < n + (4 << 30):
        pytest.skip("needs %.1f GB of free device memory" % ((n + (4 << 30)) / 1e9))
    data = inputs.stream_bytes_torch(41, 0, n, dev)
    ref = oracle.seed_expand(7, oracle.seed_words(width, b))
    h = Hasher(code, seed_words=abi.ht_seed_expand(7, code))
    got = h.hash(data).cpu().numpy().view(np.uint64)
    h.status()
    host = data.cpu().numpy()
    del data
    want, counts = oracle.hash_bytes(width, ref, host, b=b, level_counts=True)
    assert counts[:9] == [3, 0, 0, 0, 5, 0, 0, 1, 1]
    assert np.array_equal(got, want)
    h.close()


def test_parts_of_a_deep_string(dev):
    """The same deep string (512-bit blocks) hashed as three parts cut inside
    groups of levels 6 and 7, the part states merged: the digest equals the
    one-shot digest (checked against the oracle above for this length) and
    the incremental digest over uneven pieces."""
    from paper_2104_08865_gb300 import Hasher, abi
    width = 40
    xb = oracle.params(width)["exec_bytes"]
    N = 8**8 + 8**7 + 5 * 8**4 + 3
    n = N * xb + xb // 2 + 37
    free, _ = torch.cuda.mem_get_info()
    if free < n + (4 << 30):
        pytest.skip("needs %.1f GB of free device memory" % ((n + (4 << 30)) / 1e9))
    data = inputs.stream_bytes_torch(41, 0, n, dev)
    seeds = abi.ht_seed_expand(7, width)
    whole = Hasher(width, seed_words=seeds)
    want = whole.hash(data).cpu().numpy().view(np.uint64)
    parts = [Hasher(width, seed_words=seeds) for _ in range(3)]
    gran = abi.ht_part_granule(whole.ctx)
    chunks = n // gran
    cuts = [0, (3 * 8**5 + 5 * 8**3 + 1) * gran, (chunks // 8**5 - 2) * 8**5 * gran + 17 * gran, n]
    for h in parts:
        abi.ht_part_begin(h.ctx, n)
    for i in range(3):
        abi.ht_hash_part(parts[i].ctx, data.data_ptr() + cuts[i], cuts[i], cuts[i + 1] - cuts[i])
    for i in (1, 2):
        ptr, words = abi.ht_part_state(parts[i].ctx)
        abi.ht_part_merge(parts[0].ctx, ptr, words)
    got = torch.empty(width // 8, dtype=torch.int64, device=dev)
    abi.ht_finish_parts(parts[0].ctx, got.data_ptr())
    for h in parts:
        h.status()
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)
    inc = abi.ht_inc_create(whole.ctx)
    o, step = 0, 3_000_000_017
    while o < n:
        m = min(step, n - o)
        abi.ht_inc_update(inc, data.data_ptr() + o, m)
        o += m
    abi.ht_inc_final(inc, got.data_ptr())
    abi.ht_inc_status(inc)
    abi.ht_inc_destroy(inc)
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)
    for h in parts + [whole]:
        h.close()
