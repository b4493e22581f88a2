"""Long strings in the device table by their digests: deduplication and join
by content, bit-exact against the oracle (digests from the oracle's
HalftimeHash, representatives and finds from their plain definitions), and,
as a check of the whole chain, against plain byte equality of the strings.
The batches mix distinct strings, exact copies at other addresses, near
copies (one byte changed), empty strings and many copies of one string."""
import numpy as np
import pytest

import oracle
from oracle import compose
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
    return Hasher(width, seed_words=abi.ht_seed_expand(seed, width)), oracle.seed_expand(seed, oracle.seed_words(width))


def _u32(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


def _strings(seed, n_distinct, n_copies, n_near, n_empty, rng):
    """A list of byte strings: distinct slices of a splitmix64 stream, exact
    copies of some of them, near copies (one byte changed) and empties, in a
    shuffled order."""
    lens = inputs.log_uniform_lengths(seed, n_distinct, 16, 64 << 10)
    offs = np.concatenate([[0], np.cumsum(lens)])
    src = inputs.stream_bytes(seed, 0, int(offs[-1]))
    out = [src[offs[i]:offs[i] + lens[i]].copy() for i in range(n_distinct)]
    for _ in range(n_copies):
        out.append(out[int(rng.integers(0, n_distinct))].copy())
    for _ in range(n_near):
        s = out[int(rng.integers(0, n_distinct))].copy()
        s[int(rng.integers(0, len(s)))] ^= 1 + int(rng.integers(0, 255))
        out.append(s)
    out += [np.zeros(0, dtype=np.uint8) for _ in range(n_empty)]
    perm = rng.permutation(len(out))
    return [out[i] for i in perm]


def _pack(strings, dev):
    offs = []
    pos = 0
    for s in strings:
        offs.append(pos)
        pos += (len(s) + 255) // 256 * 256
    buf = np.zeros(max(pos, 256), dtype=np.uint8)
    for o, s in zip(offs, strings):
        buf[o:o + len(s)] = s
    lens = np.array([len(s) for s in strings], dtype=np.int64)
    dbuf = torch.from_numpy(buf).to(dev)
    ptrs = torch.tensor([dbuf.data_ptr() + o for o in offs], dtype=torch.int64, device=dev)
    return buf, np.array(offs), lens, dbuf, ptrs, torch.tensor(lens, dtype=torch.int64, device=dev)


def _byte_reps(strings, first=0, seen=None):
    seen = {} if seen is None else seen
    out = []
    for i, s in enumerate(strings):
        out.append(seen.setdefault(s.tobytes(), first + i))
    return np.array(out, dtype=np.uint32)


@pytest.mark.parametrize("width", WIDTHS)
def test_dedup_and_join_match_oracle(dev, width):
    from paper_2104_08865_gb300 import Table
    h, ref = _pair(width)
    rng = np.random.default_rng(100 + width)
    a = _strings(31, 1500, 400, 200, 5, rng)
    buf, offs, lens, dbuf, ptrs, lt = _pack(a, dev)
    dig = h.hash_batch(ptrs, lt, len(a))
    want_dig = oracle.hash_many(width, ref, buf, offs, lens)
    torch.cuda.synchronize()
    assert np.array_equal(dig.cpu().numpy().view(np.uint64), want_dig)
    seen = {}
    want_rep = compose.representatives(want_dig, 0, seen)
    assert np.array_equal(want_rep, _byte_reps(a))  # no digest collision among these strings
    with Table(h, max_entries=4000, seed64=99) as t:
        assert np.array_equal(_u32(t.insert(dig)), want_rep)
        assert t.entries() == len(a)
        # a second batch: ids continue, representatives may be earlier entries
        b = _strings(32, 300, 100, 50, 2, rng) + [a[i] for i in rng.integers(0, len(a), 200)]
        buf2, offs2, lens2, dbuf2, ptrs2, lt2 = _pack(b, dev)
        dig2 = h.hash_batch(ptrs2, lt2, len(b))
        want_dig2 = oracle.hash_many(width, ref, buf2, offs2, lens2)
        want_rep2 = compose.representatives(want_dig2, len(a), seen)
        assert np.array_equal(_u32(t.insert(dig2)), want_rep2)
        # joins: strings from both batches and new ones
        c = [b[i] for i in rng.integers(0, len(b), 100)] + _strings(33, 200, 0, 0, 0, rng)
        buf3, offs3, lens3, dbuf3, ptrs3, lt3 = _pack(c, dev)
        dig3 = h.hash_batch(ptrs3, lt3, len(c))
        want3 = compose.find(oracle.hash_many(width, ref, buf3, offs3, lens3), seen)
        assert np.array_equal(_u32(t.find(dig3)), want3)
        assert (want3 != compose.NOT_FOUND).sum() >= 100
        t.status()
        t.clear()
        assert t.entries() == 0
        assert np.all(_u32(t.find(dig3)) == compose.NOT_FOUND)


def test_many_copies_and_a_full_table(dev):
    """One string 3000 times among 1000 others in a table sized exactly for
    them (half full): every copy's representative is the first copy."""
    from paper_2104_08865_gb300 import HalftimeError, Table, abi
    width = 32
    h, ref = _pair(width)
    rng = np.random.default_rng(5)
    base = _strings(34, 1000, 0, 0, 0, rng)
    one = base[17]
    a = list(base) + [one.copy() for _ in range(3000)]
    a = [a[i] for i in rng.permutation(len(a))]
    buf, offs, lens, dbuf, ptrs, lt = _pack(a, dev)
    dig = h.hash_batch(ptrs, lt, len(a))
    want = compose.representatives(oracle.hash_many(width, ref, buf, offs, lens))
    with Table(h, max_entries=len(a), seed64=1) as t:
        got = _u32(t.insert(dig))
        assert np.array_equal(got, want)
        first = min(i for i, s in enumerate(a) if s.tobytes() == one.tobytes())
        assert all(got[i] == first for i, s in enumerate(a) if s.tobytes() == one.tobytes())
        # no room for more: refused before any GPU work, nothing inserted
        with pytest.raises(HalftimeError) as e:
            t.insert(dig[:1])
        assert e.value.code == abi.HT_ERR_BUDGET
        assert t.entries() == len(a)
        t.status()


def test_dedup_of_the_50000_string_batch(dev):
    """The 50,000-string batch (log-uniform 64 B .. 1 MiB) plus 12,500 entries
    that alias earlier strings' bytes: the representatives are what the
    construction fixes (the first occurrence), checked without any GPU
    digest as reference."""
    from paper_2104_08865_gb300 import Table
    width = 24
    h, _ = _pair(width)
    lens = inputs.log_uniform_lengths(3, 50_000, 64, 1 << 20)
    offs = np.zeros(len(lens), dtype=np.int64)
    offs[1:] = np.cumsum((lens[:-1] + 255) // 256 * 256)
    total = int(offs[-1] + lens[-1])
    dbuf = inputs.stream_bytes_torch(3, 0, total + 256, dev)
    rng = np.random.default_rng(8)
    alias = rng.integers(0, len(lens), 12_500)
    all_offs = np.concatenate([offs, offs[alias]])
    all_lens = np.concatenate([lens, lens[alias]])
    ptrs = torch.tensor(dbuf.data_ptr() + all_offs, dtype=torch.int64, device=dev)
    lt = torch.tensor(all_lens, dtype=torch.int64, device=dev)
    h_res = h.hash_batch(ptrs, lt, len(all_lens))
    with Table(h, max_entries=len(all_lens), seed64=3) as t:
        rep = _u32(t.insert(h_res)).astype(np.int64)
    # distinct slices of a random stream are distinct strings: each original
    # is its own representative, each alias maps to its original
    assert np.array_equal(rep[:len(lens)], np.arange(len(lens)))
    assert np.array_equal(rep[len(lens):], alias)
