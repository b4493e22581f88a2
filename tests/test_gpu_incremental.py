"""Incremental hashing (init / update / final): a string fed in pieces of any
length, from device or host memory, gives bit for bit the oracle's digest of
the whole string, however it is cut; saved states resume in another handle.
The cuts cover pieces inside one chunk, pieces that straddle chunks, whole
chunks from unaligned addresses, and strings deep enough (several hundred
chunks) that pending groups of levels 3 to 5 are completed by a later update
than the one that started them."""
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
    return Hasher(width, seed_words=abi.ht_seed_expand(seed, width)), oracle.seed_expand(seed, oracle.seed_words(width))


def _u64(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def _cuts(kind, n, gran, rng):
    """Piece lengths (some zero) that add up to n."""
    if kind == "whole":
        return [n]
    if kind == "granules":
        return [gran] * (n // gran) + [n % gran]
    out = []
    left = n
    while left:
        if kind == "small":
            p = int(rng.integers(1, gran // 3))
        else:  # mixed
            p = int(rng.choice([0, 1, 7, gran - 1, gran, gran + 1, 3 * gran + 5,
                                int(rng.integers(1, 40 * gran))]))
        p = min(p, left)
        out.append(p)
        left -= p
    return out


def _feed(inc, dbuf, host, pieces, host_every=0):
    off = 0
    for i, p in enumerate(pieces):
        if host_every and i % host_every == 1:
            inc.update(host[off:off + p])
        else:
            inc.update(dbuf[off:off + p])
        off += p
    assert inc.length() == off


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("kind", ["whole", "granules", "small", "mixed"])
def test_pieces_match_oracle(dev, width, kind):
    h, ref = _pair(width)
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    n = 587 * gran + 13 * xb + 101  # levels up to 5; remainder: 13 executions + tail
    dbuf = inputs.stream_bytes_torch(21, 0, n, dev)
    host = dbuf.cpu().numpy()
    want = oracle.hash_bytes(width, ref, host)
    rng = np.random.default_rng(1000 + width)
    with h.incremental() as inc:
        assert inc.granule() == gran
        _feed(inc, dbuf, host, _cuts(kind, n, gran, rng))
        assert np.array_equal(_u64(inc.final()), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_host_and_device_pieces_mixed(dev, width):
    h, ref = _pair(width)
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    n = 1500 * gran + 5 * xb + 3  # host pieces longer than one staging slot too
    dbuf = inputs.stream_bytes_torch(22, 0, n, dev)
    host = dbuf.cpu().numpy()
    pinned = torch.empty(n, dtype=torch.uint8).pin_memory()
    pinned.copy_(torch.from_numpy(host))
    want = oracle.hash_bytes(width, ref, host)
    rng = np.random.default_rng(2000 + width)
    pieces = [1234 * gran + 17] + _cuts("mixed", n - 1234 * gran - 17, gran, rng)
    with h.incremental() as inc:
        inc.update(pinned.numpy()[:pieces[0]])  # one long host piece first
        off = pieces[0]
        for i, p in enumerate(pieces[1:]):
            inc.update(host[off:off + p] if i % 2 else dbuf[off:off + p])
            off += p
        assert np.array_equal(_u64(inc.final()), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_short_strings_byte_by_byte(dev, width):
    h, ref = _pair(width)
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    src = inputs.stream_bytes_torch(23, 0, gran + 9, dev)
    host = src.cpu().numpy()
    with h.incremental() as inc:
        for n in (0, 1, 7, 8, 9, xb - 1, xb, xb + 1, 2 * xb + 40, gran - 1, gran, gran + 1, gran + 9):
            inc.init()
            step = 1 if n <= 2 * xb + 40 else 997
            for o in range(0, n, step):
                inc.update(src[o:min(n, o + step)])
            assert np.array_equal(_u64(inc.final()), oracle.hash_bytes(width, ref, host[:n])), n


@pytest.mark.parametrize("width", [24, 40])
def test_saved_state_resumes_in_another_handle(dev, width):
    from paper_2104_08865_gb300 import HalftimeError
    h, ref = _pair(width)
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    n = 300 * gran + 40 * xb + 77
    dbuf = inputs.stream_bytes_torch(24, 0, n, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    cut = 141 * gran + 3 * xb + 5  # inside a chunk and inside level-3/4 groups
    a = h.incremental()
    a.update(dbuf[:cut])
    state = a.export_state()
    b = h.incremental()
    b.import_state(state)
    assert b.length() == cut
    b.update(dbuf[cut:])
    a.update(dbuf[cut:])
    assert np.array_equal(_u64(b.final()), want)
    assert np.array_equal(_u64(a.final()), want)
    # another width, other seed words, a short buffer: refused
    other_w, _ = _pair(16 if width != 16 else 24)
    with pytest.raises(HalftimeError):
        other_w.incremental().import_state(state)
    other_s, _ = _pair(width, seed=8)
    with pytest.raises(HalftimeError):
        other_s.incremental().import_state(state)
    with pytest.raises(HalftimeError):
        b.import_state(state[:100])
    # a closed string takes no updates until init
    with pytest.raises(HalftimeError):
        a.update(dbuf[:10])
    a.init()
    a.update(dbuf[:10])
    assert np.array_equal(_u64(a.final()), oracle.hash_bytes(width, ref, dbuf[:10].cpu().numpy()))
    a.close()
    b.close()


def test_handles_on_two_streams_are_independent(dev):
    width = 32
    h, ref = _pair(width)
    gran = 64 * oracle.params(width)["exec_bytes"]
    n1, n2 = 200 * gran + 999, 170 * gran + 5
    d1 = inputs.stream_bytes_torch(25, 0, n1, dev)
    d2 = inputs.stream_bytes_torch(26, 0, n2, dev)
    want1 = oracle.hash_bytes(width, ref, d1.cpu().numpy())
    want2 = oracle.hash_bytes(width, ref, d2.cpu().numpy())
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    a, b = h.incremental(), h.incremental()
    rng = np.random.default_rng(5)
    c1 = _cuts("mixed", n1, gran, rng)
    c2 = _cuts("mixed", n2, gran, rng)
    o1 = o2 = 0
    for i in range(max(len(c1), len(c2))):
        if i < len(c1):
            a.update(d1[o1:o1 + c1[i]], stream=s1)
            o1 += c1[i]
        if i < len(c2):
            b.update(d2[o2:o2 + c2[i]], stream=s2)
            o2 += c2[i]
    out1 = torch.empty(4, dtype=torch.int64, device=dev)
    out2 = torch.empty(4, dtype=torch.int64, device=dev)
    a.final(out1, stream=s1)
    b.final(out2, stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(out1), want1)
    assert np.array_equal(_u64(out2), want2)


@pytest.mark.parametrize("width", [24, 40])
def test_one_gib_string_in_pieces(dev, width):
    """The 1 GiB string of the benchmark (splitmix64(2) bytes) fed in pieces
    of up to 200 MB (deep levels completed across updates) equals the
    oracle's digest and the one-shot kernel's."""
    h, ref = _pair(width)
    n = 1 << 30
    dbuf = inputs.stream_bytes_torch(2, 0, n, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    rng = np.random.default_rng(7)
    pieces = []
    left = n
    while left:
        p = min(left, int(rng.integers(1, 200 << 20)))
        pieces.append(p)
        left -= p
    with h.incremental() as inc:
        _feed(inc, dbuf, None, pieces)
        assert np.array_equal(_u64(inc.final()), want)
    assert np.array_equal(_u64(h.hash(dbuf)), want)


def test_update_longer_than_one_launch(dev):
    """One update of more than 65536 chunks (4.1 GB at width 40) runs as
    several launches; the digest equals the oracle's."""
    width = 40
    h, ref = _pair(width)
    gran = 64 * oracle.params(width)["exec_bytes"]
    n = 65536 * gran + 1000 * gran + 12345
    dbuf = inputs.stream_bytes_torch(27, 0, n, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    with h.incremental() as inc:
        inc.update(dbuf[:777])
        inc.update(dbuf[777:])
        assert np.array_equal(_u64(inc.final()), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_overlapped_updates_match_oracle(dev, width):
    """With HT_FLAG_OVERLAP_LAUNCHES every update kernel (and the kernel that
    completes the buffered chunk) may start before the one before it has
    ended; pieces that straddle chunks back to back, without a host
    synchronisation, and a piece above 32 MiB (the warp-chunk update kernel)
    still give the oracle's digest, and the handle's status stays clean."""
    from paper_2104_08865_gb300 import abi
    h, ref = _pair(width)
    abi.ht_ctx_set_flags(h.ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    big = ((33 << 20) // gran) * gran + 3 * xb + 5
    straddle = [gran - 1, gran + 1, 2 * gran + 3, 1, gran, 7, 5 * gran - 2]
    pieces = straddle * 30 + [big] + straddle * 5 + [17 * xb + 9]
    n = sum(pieces)
    dbuf = inputs.stream_bytes_torch(28, 0, n, dev)
    want = oracle.hash_bytes(width, ref, dbuf.cpu().numpy())
    with h.incremental() as inc:
        for rep in range(2):
            inc.init()
            _feed(inc, dbuf, None, pieces)
            assert np.array_equal(_u64(inc.final()), want), rep
        inc.status()


def test_overlapped_updates_between_one_shot_hashes(dev):
    """Overlapping update kernels interleaved with overlapping one-shot hashes
    of the same context on one stream: both kinds keep their digests."""
    from paper_2104_08865_gb300 import abi
    width = 32
    h, ref = _pair(width)
    abi.ht_ctx_set_flags(h.ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
    gran = 64 * oracle.params(width)["exec_bytes"]
    pieces = [3 * gran + 11, 5 * gran - 11, 1, 200 * gran + 99, gran - 100, 4000 * gran + 3, 2]
    n = sum(pieces)
    dbuf = inputs.stream_bytes_torch(29, 0, n, dev)
    host = dbuf.cpu().numpy()
    want = oracle.hash_bytes(width, ref, host)
    one_shot = [(0, 5 * gran + 1), (gran + 3, 300 * gran), (7, 2 * gran)]
    want_one = [oracle.hash_bytes(width, ref, host[o:o + m]) for o, m in one_shot]
    outs = torch.empty((len(pieces), len(one_shot), h.k), dtype=torch.int64, device=dev)
    with h.incremental() as inc:
        off = 0
        for i, p in enumerate(pieces):
            inc.update(dbuf[off:off + p])
            off += p
            for j, (o, m) in enumerate(one_shot):
                h.hash(dbuf, m, out=outs[i, j], offset=o)
        got = _u64(inc.final())
        inc.status()
    h.status()
    assert np.array_equal(got, want)
    all_one = outs.cpu().numpy().view(np.uint64)
    for i in range(len(pieces)):
        for j in range(len(one_shot)):
            assert np.array_equal(all_one[i, j], want_one[j]), (i, j)
