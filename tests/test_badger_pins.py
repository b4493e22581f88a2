"""Pins of the oracle's binary-tree ablation (Badger's approach, Section 5.2:
Carter and Wegman's tree T of Eq. algebraic-badger consumes the EHC outputs
whole, with no pending roots and no final NH).

The oracle evaluates T by its top-down recursion.  These tests check it
against things other than that recursion: T written out by hand for one to
seven leaves, a bottom-up evaluation of complete trees combined by the
binary digits of the leaf count (a closed form derived from the equation:
every complete subtree but the last enters through NH under the key of its
height, the last one unhashed), the default hash at b = 1, f = 2 (whose
complete trees the brute-force pins of test_oracle_pins.py fix), the empty
string, seed-region boundaries and lane order.
"""
import random

import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
BLEVELS = 64


def _nh(x, s):
    return (((x + s) & M32) * (((x >> 32) + (s >> 32)) & M32)) & M64


def _layout(width, b=8):
    p = oracle.params(width)
    T = p["e"] * p["w"]
    R = T + p["k"] * BLEVELS
    return dict(T=T, R=R, total=R + b * p["d"] * p["w"] + p["k"])


def _seeds(width, seed, b=8):
    return oracle.seed_expand(seed, oracle.seed_words_badger(width, b))


def _leaves(width, seeds, data, N, b):
    """EHC outputs (oracle EHC, pinned in test_oracle_pins.py) in leaf order:
    execution-major, lane-minor."""
    xb = 8 * b * oracle.params(width)["d"] * 3
    out = []
    for x in range(N):
        for lane in range(b):
            out.append([int(v) for v in oracle.ehc(width, seeds, data[x * xb:(x + 1) * xb], lane=lane, b=b)])
    return out


def _tail(S, R, t, data, n, N, xb):
    tail = bytes(data[N * xb:n])
    words = [int.from_bytes(tail[i:i + 8].ljust(8, b"\0"), "little") for i in range(0, len(tail), 8)] + [n]
    acc = 0
    for m, wd in enumerate(words):
        acc = (acc + _nh(wd, S[R + t + m])) & M64
    return acc


def _by_hand(k, y):
    """T of Eq. algebraic-badger for 1..7 leaves, written out."""
    H = lambda i, a, b: (_nh(a, k[i]) + b) & M64
    n = len(y)
    if n == 1:
        return y[0]
    if n == 2:
        return H(0, y[0], y[1])
    if n == 3:
        return H(1, H(0, y[0], y[1]), y[2])
    t4 = H(1, H(0, y[0], y[1]), H(0, y[2], y[3]))
    if n == 4:
        return t4
    if n == 5:
        return H(2, t4, y[4])
    if n == 6:
        return H(2, t4, H(0, y[4], y[5]))
    return H(2, t4, H(1, H(0, y[4], y[5]), y[6]))


def _complete_bottom_up(k, y):
    """A complete tree over 2^a leaves, level by level from the leaves."""
    level = list(y)
    h = 0
    while len(level) > 1:
        level = [(_nh(level[2 * i], k[h]) + level[2 * i + 1]) & M64 for i in range(len(level) // 2)]
        h += 1
    return level[0]


def _by_digits(k, y):
    """Closed form of Eq. algebraic-badger: split the n leaves into complete
    trees of 2^a leaves, one per set bit a of n, largest first; all but the
    last enter as NH(root, k_a), the last one unhashed."""
    n = len(y)
    bits = [a for a in range(64) if (n >> a) & 1][::-1]
    acc, pos = 0, 0
    for j, a in enumerate(bits):
        c = _complete_bottom_up(k, y[pos:pos + (1 << a)])
        pos += 1 << a
        acc = (acc + (c if j == len(bits) - 1 else _nh(c, k[a]))) & M64
    return acc


def test_seed_layout():
    for w in (16, 24, 32, 40):
        for b in (1, 4, 8):
            assert oracle.seed_words_badger(w, b) == _layout(w, b)["total"]


@pytest.mark.parametrize("width", [16, 24, 40])
def test_by_hand_b1(width):
    """b = 1, one to seven executions: the oracle equals T written out by hand
    plus the Toeplitz tail."""
    b = 1
    xb = 8 * b * oracle.params(width)["d"] * 3
    seeds = _seeds(width, 31, b)
    S = [int(v) for v in seeds]
    L = _layout(width, b)
    data = inputs.stream_bytes(17, 0, 8 * xb)
    k_ = oracle.params(width)["k"]
    for N in range(1, 8):
        for extra in (0, 13):
            n = N * xb + extra
            got = oracle.hash_bytes_badger(width, seeds, data[:n], b=b)
            lv = _leaves(width, seeds, data, N, b)
            for t in range(k_):
                keys = S[L["T"] + BLEVELS * t:L["T"] + BLEVELS * (t + 1)]
                want = (_by_hand(keys, [v[t] for v in lv]) + _tail(S, L["R"], t, data, n, N, xb)) & M64
                assert int(got[t]) == want, (width, N, extra, t)


@pytest.mark.parametrize("width,b", [(24, 8), (40, 8), (16, 4), (32, 2), (24, 3)])
def test_digit_decomposition(width, b):
    """Any leaf count: the oracle equals the closed form by binary digits
    (complete trees evaluated bottom-up)."""
    xb = 8 * b * oracle.params(width)["d"] * 3
    seeds = _seeds(width, 5 + b, b)
    S = [int(v) for v in seeds]
    L = _layout(width, b)
    rng = random.Random(width * 10 + b)
    Ns = [1, 2, 3, 5, 7, 8, 9, 15, 16, 17, 24, 31, 33] + [rng.randrange(1, 70) for _ in range(4)]
    data = inputs.stream_bytes(19, 0, 71 * xb)
    k_ = oracle.params(width)["k"]
    for N in Ns:
        n = N * xb + rng.randrange(0, xb)
        got = oracle.hash_bytes_badger(width, seeds, data[:n], b=b)
        lv = _leaves(width, seeds, data, N, b)
        for t in range(k_):
            keys = S[L["T"] + BLEVELS * t:L["T"] + BLEVELS * (t + 1)]
            want = (_by_digits(keys, [v[t] for v in lv]) + _tail(S, L["R"], t, data, n, N, xb)) & M64
            assert int(got[t]) == want, (width, b, N, t)


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_complete_trees_match_default_hash(width):
    """b = 1, f = 2, N = 2^a executions, no tail bytes: the default hash keeps
    one pending root, the complete tree over all leaves, and adds its NH under
    F[t][a][0][0]; the ablation adds the same tree unhashed.  With the default
    layout's tree keys copied into the ablation's level keys, the two agree
    after that final NH."""
    b, f, LV = 1, 2, 19
    p = oracle.params(width)
    xb = 8 * b * p["d"] * 3
    sd = oracle.seed_expand(41, oracle.seed_words(width, b, f))
    Td = p["e"] * 3
    Fd = Td + p["k"] * LV * (f - 1)
    Rd = Fd + p["k"] * LV * f * b
    sb = _seeds(width, 43, b)
    L = _layout(width, b)
    sb[:Td] = sd[:Td]  # same EHC keys
    for t in range(p["k"]):
        for lv in range(LV):
            sb[L["T"] + BLEVELS * t + lv] = sd[Td + t * LV + lv]
    data = inputs.stream_bytes(23, 0, 64 * xb)
    for a in range(0, 7):
        N = 1 << a
        n = N * xb
        dd = oracle.hash_bytes(width, sd, data[:n], b=b, f=f)
        db = oracle.hash_bytes_badger(width, sb, data[:n], b=b)
        for t in range(p["k"]):
            tree = (int(db[t]) - _nh(n, int(sb[L["R"] + t]))) & M64
            want = (_nh(tree, int(sd[Fd + (t * LV + a) * f])) + _nh(n, int(sd[Rd + t]))) & M64
            assert int(dd[t]) == want, (width, a, t)


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_empty_and_tail_only(width):
    """Without a whole execution there are no leaves: the digest is the
    Toeplitz tail with the length word alone; the empty string gives
    NH(0, R[t])."""
    seeds = _seeds(width, 3)
    S = [int(v) for v in seeds]
    L = _layout(width)
    xb = oracle.params(width)["exec_bytes"]
    got = oracle.hash_bytes_badger(width, seeds, b"")
    for t in range(oracle.params(width)["k"]):
        assert int(got[t]) == ((S[L["R"] + t] & M32) * (S[L["R"] + t] >> 32)) & M64
    data = inputs.stream_bytes(29, 0, xb)
    for n in (1, 8, 9, 100, xb - 1):
        got = oracle.hash_bytes_badger(width, seeds, data[:n])
        for t in range(oracle.params(width)["k"]):
            assert int(got[t]) == _tail(S, L["R"], t, data, n, 0, xb)


def test_level_keys_used_exactly():
    """N executions at b = 8 give 8N leaves, so T reads k_0 .. k_{ceil(lg 8N)-1}
    of each tree and no higher key; EHC keys and tail keys are read too."""
    width = 24
    p = oracle.params(width)
    L = _layout(width)
    xb = p["exec_bytes"]
    data = inputs.stream_bytes(37, 0, 6 * xb)
    base = _seeds(width, 9)
    n = 5 * xb + 40  # 40 leaves: keys 0..5
    d0 = oracle.hash_bytes_badger(width, base, data[:n])
    for t in range(p["k"]):
        for i in (0, 3, 5, 6, 7, 40):
            s = base.copy()
            s[L["T"] + BLEVELS * t + i] ^= np.uint64(1 << 40)
            changed = not np.array_equal(oracle.hash_bytes_badger(width, s, data[:n]), d0)
            assert changed == (i <= 5), (t, i)
    for j in (0, p["e"] * 3 - 1, L["R"], L["R"] + p["k"] + 4):  # tail words m = 0..5
        s = base.copy()
        s[j] ^= np.uint64(1 << 33)
        assert not np.array_equal(oracle.hash_bytes_badger(width, s, data[:n]), d0), j


def test_lane_order():
    """Leaves are lane-minor: swapping the contents of lanes 0 and 1 of one
    execution changes the digest (the two leaves sit in one height-1 node,
    left hashed, right not), and the by-hand T over leaves in lane-minor order
    matches at b = 2, N = 1..3."""
    width, b = 16, 2
    p = oracle.params(width)
    xb = 8 * b * p["d"] * 3
    seeds = _seeds(width, 47, b)
    S = [int(v) for v in seeds]
    L = _layout(width, b)
    data = inputs.stream_bytes(53, 0, 3 * xb)
    for N in (1, 2, 3):
        n = N * xb
        got = oracle.hash_bytes_badger(width, seeds, data[:n], b=b)
        lv = _leaves(width, seeds, data, N, b)
        for t in range(p["k"]):
            keys = S[L["T"] + BLEVELS * t:L["T"] + BLEVELS * (t + 1)]
            want = (_by_hand(keys, [v[t] for v in lv]) + _tail(S, L["R"], t, data, n, N, xb)) & M64
            assert int(got[t]) == want
    sw = np.array(data[:xb], dtype=np.uint8).reshape(-1, b, 8)[:, ::-1, :].reshape(-1)
    assert not np.array_equal(oracle.hash_bytes_badger(width, seeds, sw.tobytes(), b=b),
                              oracle.hash_bytes_badger(width, seeds, data[:xb], b=b))
