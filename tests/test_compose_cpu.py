"""The short-input hash that keys the digest table (vector multiply-shift over
a digest's 32-bit halves) and the table's deduplication semantics, on the CPU:
the oracle's definitions are pinned by closed forms, by the strong
universality of the bits the table uses (and the failure of the bits it does
not use), and by hand-worked examples; the library's host form of the hash
and its key expansion equal the oracle's."""
import numpy as np
import pytest

from oracle import compose

MASK64 = (1 << 64) - 1


def _rand_u64(rng, n):
    return [int(v) for v in rng.integers(0, 2**64, size=n, dtype=np.uint64)]


def _rand_digest(rng, k):
    return _rand_u64(rng, k)


def test_slot_hash_closed_forms():
    rng = np.random.default_rng(1)
    for k in (2, 3, 4, 5):
        d = _rand_digest(rng, k)
        zero = [0] * (2 * k + 1)
        c = 0x0123456789ABCDEF
        assert compose.slot_hash([c] + zero[1:], d) == c
        for i in range(k):
            lo = zero.copy()
            lo[1 + 2 * i] = 1
            hi = zero.copy()
            hi[2 + 2 * i] = 1
            assert compose.slot_hash(lo, d) == d[i] & 0xFFFFFFFF
            assert compose.slot_hash(hi, d) == d[i] >> 32
        # keys 1 and 2^32 on the halves of every word rebuild the words: h = a_0 + sum of words
        keys = [7] + [1, 1 << 32] * k
        assert compose.slot_hash(keys, d) == (7 + sum(d)) & MASK64


def _chi2_pairs(x, y, bits, top, n=16384, seed=3):
    """Chi-square of the joint distribution of `bits` output bits of h(x) and
    h(y) over n random key sets (top or low bits), against uniform."""
    rng = np.random.default_rng(seed)
    k = len(x)
    cells = np.zeros((1 << bits, 1 << bits), dtype=np.int64)
    for _ in range(n):
        keys = _rand_u64(rng, 2 * k + 1)
        hx, hy = compose.slot_hash(keys, x), compose.slot_hash(keys, y)
        if top:
            hx, hy = hx >> (64 - bits), hy >> (64 - bits)
        else:
            hx, hy = hx & ((1 << bits) - 1), hy & ((1 << bits) - 1)
        cells[hx, hy] += 1
    exp = n / cells.size
    return float(((cells - exp) ** 2 / exp).sum())


def test_top_bits_are_strongly_universal_low_bits_are_not():
    # digests differing only in bit 31 of the first 32-bit half: h(x) - h(y)
    # = a_1 2^31 mod 2^64, so the low 31 bits of h(x) and h(y) always agree
    x = [0x1111111122222222, 0x3333333344444444]
    y = [x[0] ^ (1 << 31), x[1]]
    top = _chi2_pairs(x, y, bits=2, top=True)
    low = _chi2_pairs(x, y, bits=2, top=False)
    assert top < 37.7, top   # 15 degrees of freedom, p = 0.001
    assert low > 1000, low   # mass only on the diagonal
    # a pair differing in a high half of a later word, five words
    rng = np.random.default_rng(9)
    x5 = _rand_digest(rng, 5)
    y5 = list(x5)
    y5[3] ^= 1 << 60
    assert _chi2_pairs(x5, y5, bits=2, top=True, n=8192, seed=4) < 37.7


def test_representatives_and_find_by_hand():
    d = [[1, 9], [2, 9], [1, 9], [3, 9], [2, 9], [1, 8]]
    assert list(compose.representatives(d)) == [0, 1, 0, 3, 1, 5]
    seen = {}
    assert list(compose.representatives(d[:3], 0, seen)) == [0, 1, 0]
    assert list(compose.representatives(d[3:], 3, seen)) == [3, 1, 5]
    assert list(compose.find([[2, 9], [4, 9], [1, 8]], seen)) == [1, compose.NOT_FOUND, 5]


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_library_short_hash_matches_oracle(built, width):
    from paper_2104_08865_gb300 import abi
    k = width // 8
    for seed in (0, 7, 2**64 - 1):
        keys = abi.ht_short_hash_keys(seed, width)
        assert [int(v) for v in keys] == compose.table_keys(seed, k)
    rng = np.random.default_rng(width)
    keys = compose.table_keys(12345, k)
    for _ in range(200):
        d = _rand_digest(rng, k)
        assert abi.ht_short_hash(np.array(keys, dtype=np.uint64), width,
                                 np.array(d, dtype=np.uint64)) == compose.slot_hash(keys, d)
    with pytest.raises(abi.HalftimeError):
        abi.ht_short_hash_keys(1, 17)
