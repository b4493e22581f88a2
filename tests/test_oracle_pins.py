"""Pins of the CPU oracle against facts the paper or mathematics fixes.

Each test checks the oracle against something other than itself: numbers the
paper prints (tests/golden/), closed forms, invariants, exhaustive
enumeration, or an independent brute-force evaluation of the paper's
recursive equations at tiny parameters.
"""
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
LEVELS = 19


def _golden_matrices():
    mats = {}
    cur = None
    for line in open(os.path.join(GOLDEN, "combine_matrices.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "width":
            cur = int(tok[1])
            mats[cur] = {"p": int(tok[3]), "T": []}
        else:
            mats[cur]["T"].append([int(x) for x in tok])
    return mats


def _golden_figures():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_figures.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            tok = line.split()
            out[tok[0]] = [float(x) for x in tok[1:]]
    return out


def _seeds(width, seed=7, b=8, f=8):
    return oracle.seed_expand(seed, oracle.seed_words(width, b, f))


def _layout(width, b=8, f=8):
    p = oracle.params(width)
    E = 0
    T = E + p["e"] * p["w"]
    F = T + p["k"] * LEVELS * (f - 1)
    R = F + p["k"] * LEVELS * f * b
    return dict(E=E, T=T, F=F, R=R, total=R + b * p["d"] * p["w"] + p["k"])


# ---------------------------------------------------------------- splitmix64

def test_splitmix64_published_outputs():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tok = [int(x) for x in line.split()]
        seed, expect = tok[0], tok[1:]
        got = oracle.seed_expand(seed, len(expect))
        assert [int(x) for x in got] == expect
        # the input generator's counter form reproduces the same stream
        assert [int(x) for x in inputs.splitmix64_words(seed, 0, len(expect))] == expect


# ------------------------------------------------------------- combine matrix

def _two_adic(n):
    n = abs(n)
    v = 0
    while n % 2 == 0:
        n //= 2
        v += 1
    return v


def _det(M):
    M = [[Fraction(x) for x in row] for row in M]
    n = len(M)
    det = Fraction(1)
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] != 0), None)
        if piv is None:
            return 0
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det *= M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            for cc in range(c, n):
                M[r][cc] -= f * M[c][cc]
    return int(det)


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_combine_matrix_minors_match_stated_p(width):
    """Section 4 theorem + Section 5.1 table: the largest power of two dividing
    any k-column minor of the printed T is the printed p; no minor is 0."""
    g = _golden_matrices()[width]
    T = g["T"]
    k, e = len(T), len(T[0])
    vmax = 0
    for cols in itertools.combinations(range(e), k):
        det = _det([[T[r][c] for c in cols] for r in range(k)])
        assert det != 0
        vmax = max(vmax, _two_adic(det))
    assert vmax == g["p"]
    p = oracle.params(width)
    assert (p["k"], p["e"]) == (k, e)
    # Section 5.1: input group length d = columns + 1 - rows
    assert p["d"] == e + 1 - k
    figs = _golden_figures()
    assert p["d"] == figs["group_lengths"][oracle.WIDTHS.index(width)]


def test_hh24_parameter_tuple():
    w, d, e, k, b, f, pexp = _golden_figures()["hh24_tuple"]
    p = oracle.params(24)
    assert (p["w"], p["d"], p["e"], p["k"]) == (w, d, e, k)
    assert p["exec_bytes"] == 8 * b * d * w
    assert _golden_matrices()[24]["p"] == pexp


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_ehc_combine_is_paper_matrix(width):
    """With all-zero data and only item c's seed word u set to (lo=1, hi=1),
    every NH term but one is 0 and that one is 1, so y = column c of T."""
    p = oracle.params(width)
    T = _golden_matrices()[width]["T"]
    ex = np.zeros(p["exec_bytes"], dtype=np.uint8)
    for c in range(p["e"]):
        for u in range(p["w"]):
            seeds = np.zeros(oracle.seed_words(width), dtype=np.uint64)
            seeds[c * p["w"] + u] = (1 << 32) | 1
            y = oracle.ehc(width, seeds, ex, lane=3)
            assert [int(v) for v in y] == [T[t][c] for t in range(p["k"])]


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_ehc_block_layout_and_nh_halves(width):
    """Word (blk = i*w + u, lane j) of an execution sits at byte 8*(blk*8 + j).
    Put x = 5 (high half 0) there; every encoded word then has a zero high
    half, so with seed (lo=0, hi=1) on data item i word u only that term
    survives: NH = (5 + 0) * (0 + 1) = 5 and y = 5 * T[:, i]."""
    p = oracle.params(width)
    T = _golden_matrices()[width]["T"]
    for i in range(p["d"]):
        for u in range(p["w"]):
            for lane in (0, 5, 7):
                ex = np.zeros(p["exec_bytes"] // 8, dtype="<u8")
                ex[(i * p["w"] + u) * 8 + lane] = 5
                seeds = np.zeros(oracle.seed_words(width), dtype=np.uint64)
                seeds[i * p["w"] + u] = 1 << 32
                y = oracle.ehc(width, seeds, ex.view(np.uint8), lane=lane)
                assert [int(v) for v in y] == [5 * T[t][i] for t in range(p["k"])]
                # another lane does not see the word
                other = (lane + 1) % 8
                y2 = oracle.ehc(width, seeds, ex.view(np.uint8), lane=other)
                assert [int(v) for v in y2] == [0] * p["k"]


# ------------------------------------------------------------- erasure codes

def _bitsliced_batches(d):
    """All 8^d vectors of GF(8) symbols, 64 per batch, as bit-sliced items:
    returns uint64 array [batches, d, 3]."""
    total = 8 ** d
    idx = np.arange(total, dtype=np.uint64).reshape(-1, 64)
    weights = (np.uint64(1) << np.arange(64, dtype=np.uint64))
    out = np.zeros((idx.shape[0], d, 3), dtype=np.uint64)
    for i in range(d):
        digit = (idx >> np.uint64(3 * i)) & np.uint64(7)
        for u in range(3):
            bit = (digit >> np.uint64(u)) & np.uint64(1)
            out[:, i, u] = (bit * weights).sum(axis=1, dtype=np.uint64)
    return out


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_code_distance_exhaustive(width):
    """Section 3.3: the code must have minimum distance k.  Enumerate every
    data vector of GF(8) symbols and count nonzero encoded items."""
    p = oracle.params(width)
    d, e, k = p["d"], p["e"], p["k"]
    batches = _bitsliced_batches(d)
    shifts = np.arange(64, dtype=np.uint64)
    best = 99
    for bi in range(batches.shape[0]):
        items = batches[bi].reshape(-1)
        enc = oracle.encode(width, items).reshape(e, 3)
        # systematic: first d items are the data
        assert np.array_equal(enc[:d], batches[bi])
        nz = enc[:, 0] | enc[:, 1] | enc[:, 2]
        bits = ((nz[:, None] >> shifts[None, :]) & np.uint64(1)).sum(axis=0)
        if bi == 0:
            bits = bits[1:]  # vector 0 is the zero vector
        best = min(best, int(bits.min()))
    assert best == k


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_code_is_linear(width):
    rng = np.random.default_rng(width)
    p = oracle.params(width)
    n = p["d"] * 3
    for _ in range(50):
        a = rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        b = rng.integers(0, 2**63, n, dtype=np.uint64)
        assert np.array_equal(oracle.encode(width, a ^ b),
                              oracle.encode(width, a) ^ oracle.encode(width, b))


# ----------------------------------------------------------------------- NH

def test_nh_closed_forms():
    rng = random.Random(1)
    for _ in range(200):
        s = rng.getrandbits(64)
        x = rng.getrandbits(64)
        # zero data: the product of the seed halves
        assert oracle.nh_word(0, s) == (s & M32) * (s >> 32)
        # low half equal to minus the seed's low half: the term vanishes
        xz = (x & ~M32 & M64) | ((-s) & M32)
        assert oracle.nh_word(xz, s) == 0
        # high half likewise
        xz = (x & M32) | ((((-(s >> 32)) & M32)) << 32)
        assert oracle.nh_word(xz, s) == 0
    # wrap-around: (2^32-1 + 1) mod 2^32 = 0
    assert oracle.nh_word(M32, 1 | (5 << 32)) == 0
    # largest product stays exact mod 2^64: (2^32-1)^2
    assert oracle.nh_word(M64, 0) == (M32 * M32) & M64


# -------------------------------------------------------------- seed budget

def test_seed_budget_matches_paper():
    """Section 6.2: e*w + (f-1)hk + bfhk + bdw + k - 1 words; the paper's
    figures are 8.4KB (1MB, h=4) and 34KB (1EB, h=19) for HalftimeHash24.
    The library layout is that budget at 19 levels plus one word of Toeplitz
    key for the length word."""
    figs = _golden_figures()
    p = oracle.params(24)
    b, f = 8, 8

    def budget(h):
        return (p["e"] * p["w"] + (f - 1) * h * p["k"] + b * f * h * p["k"]
                + b * p["d"] * p["w"] + p["k"] - 1)

    kb_small, kb_large = figs["hh24_entropy_kb"]
    assert round(budget(4) * 8 / 1000, 1) == kb_small
    assert round(budget(19) * 8 / 1000) == kb_large
    for w in oracle.WIDTHS:
        q = oracle.params(w)
        full = (q["e"] * q["w"] + (f - 1) * LEVELS * q["k"] + b * f * LEVELS * q["k"]
                + b * q["d"] * q["w"] + q["k"] - 1)
        assert oracle.seed_words(w) == full + 1
    assert [oracle.seed_words(w) for w in oracle.WIDTHS] == [2865, 4245, 5598, 6897]


def test_collision_bound_hh24():
    """Section 6.2: 2^{-32k}(2^{kp} + h^k + 1) gives > 83 bits for HH24 below
    one exabyte, with p read as the exponent 2."""
    figs = _golden_figures()
    p = oracle.params(24)
    k = p["k"]
    pexp = _golden_matrices()[24]["p"]
    n = 10 ** 18
    N = n // p["exec_bytes"]
    h = int(math.floor(math.log(N, 8)))
    bits = 32 * k - math.log2(2 ** (k * pexp) + h ** k + 1)
    assert bits > figs["hh24_output_bits_min"][0]
    # also at the full 19-level layout
    assert 32 * k - math.log2(2 ** (k * pexp) + LEVELS ** k + 1) > 83


# ---------------------------------------------------------------- tree shape

@pytest.mark.parametrize("width", [16, 40])
def test_tree_pending_roots_are_base_f_digits(width):
    """Eq. stack-construction: one complete tree per nonzero digit; with an
    eager f-ary merge the pending roots at level l number digit l of N."""
    p = oracle.params(width)
    seeds = _seeds(width)
    for N in [0, 1, 7, 8, 9, 63, 64, 65, 72, 511, 512, 585, 600]:
        data = inputs.stream_bytes(3, 0, N * p["exec_bytes"] + 17)
        _, counts = oracle.hash_bytes(width, seeds, data, level_counts=True)
        digits = []
        n = N
        for _ in range(LEVELS):
            digits.append(n % 8)
            n //= 8
        assert counts == digits


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_streaming_equals_recursive_twin(width):
    p = oracle.params(width)
    seeds = _seeds(width)
    rng = random.Random(width)
    lens = [0, 1, 8, p["exec_bytes"] - 1, p["exec_bytes"], p["exec_bytes"] + 1]
    lens += [rng.randrange(0, 80 * p["exec_bytes"]) for _ in range(12)]
    lens += [64 * p["exec_bytes"], 64 * p["exec_bytes"] + 5, 73 * p["exec_bytes"] + 100]
    data = inputs.stream_bytes(11, 0, max(lens))
    for n in lens:
        a = oracle.hash_bytes(width, seeds, data[:n])
        b = oracle.hash_bytes(width, seeds, data[:n], recursive=True)
        assert np.array_equal(a, b), n


@pytest.mark.parametrize("b,f", [(1, 2), (2, 3), (4, 5), (3, 8)])
def test_streaming_equals_recursive_debug_params(b, f):
    width = 24
    seeds = _seeds(width, 9, b, f)
    xb = 8 * b * 7 * 3
    data = inputs.stream_bytes(12, 0, (2 * f ** 3 + 4) * xb)
    for N in list(range(0, 30)) + [f ** 3 - 1, f ** 3, f ** 3 + f + 1, 2 * f ** 3 + 3]:
        n = N * xb + (N % 5) * 13
        a = oracle.hash_bytes(width, seeds, data[:n], b=b, f=f)
        r = oracle.hash_bytes(width, seeds, data[:n], b=b, f=f, recursive=True)
        assert np.array_equal(a, r), (b, f, N)


# ----------------------------------------- brute force, paper's equations

def _nh(x, s):
    return (((x + s) & M32) * ((((x >> 32) + (s >> 32)) & M32))) & M64


def _badger_T(keys, s):
    """Eq. algebraic-badger with H(k, x, y) = NH(x, k) + y (Section 3.2
    tree-node variant at fan-out 2); keys[i] is k_i."""
    n = len(s)
    if n == 1:
        return s[0]
    half = 1 << (math.ceil(math.log2(n)) - 1)
    i = math.ceil(math.log2(n) - 1)
    return (_nh(_badger_T(keys, s[:half]), keys[i]) + _badger_T(keys, s[half:])) & M64


def _stack_T(keys, s, i):
    """Eq. stack-construction, T-hat_i; returns [(level, value or None)]
    top level first.  Started at i = bit length of n, each step keeps the
    prefix of 2^(i-1) when it fits."""
    if i == 0:
        return [(0, s[0] if s else None)]
    lvl = i - 1
    if (1 << lvl) > len(s):
        return [(lvl + 1, None)] + _stack_T(keys, s, i - 1)
    return [(lvl + 1, _badger_T(keys, s[: 1 << lvl]))] + _stack_T(keys, s[1 << lvl:], i - 1)


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_bruteforce_binary_tree_b1_f2(width):
    """At b=1, f=2 evaluate the paper's recursive definitions literally in
    Python integers: EHC leaves (oracle EHC), Carter-Wegman T, the stack T-hat,
    final NH keyed per (tree, level, slot) and the Toeplitz tail with the
    length word; compare with the oracle's streaming hash."""
    p = oracle.params(width)
    b, f = 1, 2
    xb = 8 * b * p["d"] * 3
    seeds = _seeds(width, 21, b, f)
    S = [int(x) for x in seeds]
    L = _layout(width, b, f)
    rng = random.Random(width)
    data_all = inputs.stream_bytes(13, 0, 40 * xb + xb)
    for N in list(range(0, 20)) + [31, 32, 33]:
        n = N * xb + rng.randrange(0, xb)
        data = data_all[:n]
        leaves = [oracle.ehc(width, seeds, data[x * xb:(x + 1) * xb], lane=0, b=1)
                  for x in range(N)]
        out = []
        for t in range(p["k"]):
            keys = [S[L["T"] + (t * LEVELS + lv) * (f - 1)] for lv in range(LEVELS)]
            ys = [int(v[t]) for v in leaves]
            acc = 0
            if N:
                for level_plus, val in _stack_T(keys, ys, N.bit_length()):
                    if val is None:
                        continue
                    # a T of 2^(level_plus-1) leaves sits at tree level level_plus-1
                    lvl = level_plus - 1 if level_plus > 0 else 0
                    fi = L["F"] + ((t * LEVELS + lvl) * f + 0) * b + 0
                    acc = (acc + _nh(val, S[fi])) & M64
            tail = bytes(data[N * xb:])
            words = [int.from_bytes(tail[i:i + 8].ljust(8, b"\0"), "little")
                     for i in range(0, len(tail), 8)] + [n]
            for m, wd in enumerate(words):
                acc = (acc + _nh(wd, S[L["R"] + t + m])) & M64
            out.append(acc)
        got = oracle.hash_bytes(width, seeds, data, b=b, f=f)
        assert [int(v) for v in got] == out, (width, N, n)


# ----------------------------------------------------------- tail / length

@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_empty_string_closed_form(width):
    seeds = _seeds(width)
    L = _layout(width)
    got = oracle.hash_bytes(width, seeds, b"")
    k = oracle.params(width)["k"]
    want = [(int(seeds[L["R"] + t]) & M32) * (int(seeds[L["R"] + t]) >> 32) & M64
            for t in range(k)]
    assert [int(v) for v in got] == want


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_toeplitz_shift(width):
    """Section 6.1: component t of the tail hash uses r[t, bdw + t); so with
    the R region shifted left by t, component 0 reproduces component t."""
    p = oracle.params(width)
    L = _layout(width)
    seeds = _seeds(width, 31)
    rng = random.Random(width)
    for n in [0, 1, 9, 64, p["exec_bytes"] - 1]:
        data = bytes(rng.getrandbits(8) for _ in range(n))
        base = oracle.hash_bytes(width, seeds, data)
        for t in range(1, p["k"]):
            sh = seeds.copy()
            sh[L["R"]:L["total"] - t] = seeds[L["R"] + t:L["total"]]
            got = oracle.hash_bytes(width, sh, data)
            assert int(got[0]) == int(base[t])


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_lengths_separated(width):
    seeds = _seeds(width)
    seen = set()
    for n in range(0, 3000, 7):
        d = tuple(int(v) for v in oracle.hash_bytes(width, seeds, bytes(n)))
        assert d not in seen
        seen.add(d)


# --------------------------------------------------------- seed sensitivity

@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_seed_sensitivity(width):
    """Every seed word a string uses changes its digest; words it cannot use
    (slot j = f-1 of the final NH, tree levels it never reaches, Toeplitz keys
    past its tail) do not."""
    p = oracle.params(width)
    L = _layout(width)
    seeds = _seeds(width, 41)
    N = 8 * 8 + 8 + 3  # digits (3, 1, 1): levels 0, 1, 2 pending, merges at 0, 1
    tail = 40
    n = N * p["exec_bytes"] + tail
    data = inputs.stream_bytes(14, 0, n)
    base = oracle.hash_bytes(width, seeds, data)
    k = p["k"]

    def changed(idx):
        s = seeds.copy()
        s[idx] ^= np.uint64(0x1234_5678_9ABC_DEF1)
        return not np.array_equal(oracle.hash_bytes(width, s, data), base)

    for c in range(p["e"] * p["w"]):
        assert changed(L["E"] + c)
    for t in range(k):
        for lv in (0, 1):
            for i in range(7):
                assert changed(L["T"] + (t * LEVELS + lv) * 7 + i)
        assert not changed(L["T"] + (t * LEVELS + 2) * 7 + 0)
        for lv, digit in ((0, 3), (1, 1), (2, 1)):
            for j in range(8):
                idx = L["F"] + ((t * LEVELS + lv) * 8 + j) * 8 + 5
                assert changed(idx) == (j < digit)
        assert not changed(L["F"] + ((t * LEVELS + 3) * 8 + 0) * 8 + 0)
    words = (tail + 7) // 8 + 1
    for m in range(words + k - 1):
        assert changed(L["R"] + m)
    assert not changed(L["R"] + words + k - 1)


# ----------------------------------------------------------- collision rate

def test_close_pairs_do_not_collide():
    """Close pairs (one 32-bit word flipped) under fresh seeds: no collision of
    the digest, nor of any single 64-bit output word (each word alone is
    roughly 2^-30-almost-universal here, so 6,000 pairs should show none).
    Narrow windows of a word are not uniform (a changed NH term moves it by a
    product (d + s) * delta) and are not tested."""
    width = 16
    p = oracle.params(width)
    n = 2 * p["exec_bytes"] + 100
    trials = 6000
    rng = random.Random(5)
    seed_stream = inputs.splitmix64_words(11, 0, trials)
    base = inputs.stream_bytes(4, 0, n)
    for i in range(trials):
        seeds = oracle.seed_expand(int(seed_stream[i]), oracle.seed_words(width))
        x = base.copy()
        y = base.copy()
        wpos = rng.randrange(n // 4)
        flip = rng.randrange(1, 2**32)
        y[4 * wpos:4 * wpos + 4] ^= np.frombuffer(flip.to_bytes(4, "little"), np.uint8)
        a = oracle.hash_bytes(width, seeds, x)
        b = oracle.hash_bytes(width, seeds, y)
        assert not np.any(a == b), (i, wpos)


# ------------------------------------------- 256-bit blocks (b = 4, "v3")

@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_b4_block_layout_and_lanes(width):
    """With blocks of 4 words, word (blk, lane) of an execution sits at byte
    8*(blk*4 + lane) (Section 2): the probe of the 8-word layout test, at the
    4-word stride, recovers 5*T[:, i] in its own lane only."""
    p = oracle.params(width, 4)
    T = _golden_matrices()[width]["T"]
    for i in range(p["d"]):
        for u in range(p["w"]):
            for lane in range(4):
                ex = np.zeros(p["exec_bytes"] // 8, dtype="<u8")
                ex[(i * p["w"] + u) * 4 + lane] = 5
                seeds = np.zeros(oracle.seed_words(width, 4), dtype=np.uint64)
                seeds[i * p["w"] + u] = 1 << 32
                y = oracle.ehc(width, seeds, ex.view(np.uint8), lane=lane, b=4)
                assert [int(v) for v in y] == [5 * T[t][i] for t in range(p["k"])]
                y2 = oracle.ehc(width, seeds, ex.view(np.uint8), lane=(lane + 1) % 4, b=4)
                assert [int(v) for v in y2] == [0] * p["k"]


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_b4_lane_equals_b8_lane_on_restrided_words(width):
    """EHC works per lane: lane j < 4 of a 4-word-block execution equals
    lane j of the 8-word-block execution whose blocks hold the same words in
    lanes 0..3 (and anything in lanes 4..7)."""
    p4, p8 = oracle.params(width, 4), oracle.params(width, 8)
    seeds = _seeds(width)
    rng = np.random.default_rng(width)
    for _ in range(4):
        x4 = rng.integers(0, 2**64, p4["exec_bytes"] // 8, dtype=np.uint64)
        x8 = rng.integers(0, 2**64, p8["exec_bytes"] // 8, dtype=np.uint64)
        blocks = p4["d"] * p4["w"]
        x8.reshape(blocks, 8)[:, :4] = x4.reshape(blocks, 4)
        for lane in range(4):
            a = oracle.ehc(width, seeds, x4.view(np.uint8), lane=lane, b=4)
            b = oracle.ehc(width, seeds, x8.view(np.uint8), lane=lane, b=8)
            assert np.array_equal(a, b), (width, lane)


def test_b4_seed_layout():
    """Seed regions with 4-word blocks: E = e*w, T = k*19*7, F = k*19*8*4,
    R = 4*d*w + k (the layout of Section 6.2's budget at b = 4)."""
    for width in oracle.WIDTHS:
        assert oracle.seed_words(width, 4) == _layout(width, 4)["total"]
    assert [oracle.seed_words(w, 4) for w in oracle.WIDTHS] == [1577, 2337, 3082, 3797]


@pytest.mark.parametrize("width", oracle.WIDTHS)
def test_b4_streaming_equals_recursive_twin(width):
    p = oracle.params(width, 4)
    xb = p["exec_bytes"]
    seeds = _seeds(width, 7, 4)
    Ns = [0, 1, 7, 8, 63, 64, 65, 127, 128, 129, 511, 512, 513, 585, 1100]
    data = inputs.stream_bytes(14, 0, max(Ns) * xb + xb)
    for N in Ns:
        n = N * xb + (N * 37) % xb
        a = oracle.hash_bytes(width, seeds, data[:n], b=4)
        r = oracle.hash_bytes(width, seeds, data[:n], b=4, recursive=True)
        assert np.array_equal(a, r), (width, N)


def _tree_node(children, keys):
    """Section 3.2 node variant at fan-out 8: NH of the first seven children
    under the level's keys plus the eighth child."""
    acc = children[7]
    for i in range(7):
        acc += _nh(children[i], keys[i])
    return acc & M64


def _complete_tree(leaves, level, tkeys):
    """A complete 8-ary tree over 8^level leaves (node keys by height)."""
    if level == 0:
        return leaves[0]
    span = 8 ** (level - 1)
    kids = [_complete_tree(leaves[i * span:(i + 1) * span], level - 1, tkeys) for i in range(8)]
    return _tree_node(kids, tkeys[level - 1])


@pytest.mark.parametrize("width", [16, 24, 40])
def test_b4_python_evaluation(width):
    """The whole hash with 4-word blocks evaluated in Python integers from the
    oracle's EHC leaves only: complete 8-ary trees taken from the front of the
    leaf sequence, one per unit of each base-8 digit of N, highest level first
    (Eq. stack-construction with fan-out 8); final NH of root j of level l in
    lane i under F[t][l][j][i]; Toeplitz tail with the length word
    (Section 6.1)."""
    b = 4
    p = oracle.params(width, b)
    xb, k = p["exec_bytes"], p["k"]
    seeds = _seeds(width, 31, b)
    S = [int(x) for x in seeds]
    L = _layout(width, b)
    data_all = inputs.stream_bytes(15, 0, 600 * xb + xb)
    for N in [0, 3, 8, 64, 71, 130, 519, 600]:
        n = N * xb + (N * 53 + 11) % xb
        data = data_all[:n]
        leaves = [[oracle.ehc(width, seeds, data[x * xb:(x + 1) * xb], lane=i, b=b)
                   for i in range(b)] for x in range(N)]
        want = []
        for t in range(k):
            tkeys = [[S[L["T"] + (t * LEVELS + lv) * 7 + i] for i in range(7)] for lv in range(LEVELS)]
            acc = 0
            pos = 0
            for lvl in range(LEVELS - 1, -1, -1):
                span = 8 ** lvl
                j = 0
                while N - pos >= span:
                    for i in range(b):
                        ys = [int(leaves[x][i][t]) for x in range(pos, pos + span)]
                        root = _complete_tree(ys, lvl, tkeys)
                        fi = L["F"] + ((t * LEVELS + lvl) * 8 + j) * b + i
                        acc = (acc + _nh(root, S[fi])) & M64
                    pos += span
                    j += 1
            tail = bytes(data[N * xb:])
            words = [int.from_bytes(tail[i:i + 8].ljust(8, b"\0"), "little")
                     for i in range(0, len(tail), 8)] + [n]
            for m, wd in enumerate(words):
                acc = (acc + _nh(wd, S[L["R"] + t + m])) & M64
            want.append(acc)
        got = oracle.hash_bytes(width, seeds, data, b=b)
        assert [int(v) for v in got] == want, (width, N)


# ------------------------------------------------- collision rate of a window

@pytest.mark.parametrize("v,half", [(10, "lo"), (12, "hi"), (16, "lo")])
def test_tail_window_collision_rate(v, half):
    """Two strings that differ only in one tail word w -> w' = w ^ 2^v (in its
    low or high 32-bit half) differ in output word t by the difference of one
    NH term, (A)(B) - (A')(B') with one factor equal in both; the other
    factor is uniform when the data are.  Their low 16 bits then collide
    with probability exactly 2^(v-16) (v <= 16).  Count the collisions of
    out_0 over random tail-only strings under one seed and compare with that
    rate (a mistake that drops, repeats or misroutes the tail word moves the
    count far outside the band)."""
    width = 24
    xb = oracle.params(width)["exec_bytes"]
    seeds = _seeds(width, 71)
    rng = np.random.default_rng(v * 7 + (half == "hi"))
    trials = 6000 if v >= 12 else 20000
    hits = 0
    for _ in range(trials):
        n = int(rng.integers(8, xb))  # tail only: no whole execution
        data = rng.integers(0, 256, n, dtype=np.uint8)
        m = int(rng.integers(0, n // 8))  # a whole tail word
        other = data.copy()
        bit = v + (32 if half == "hi" else 0)
        other[8 * m + bit // 8] ^= np.uint8(1 << (bit % 8))
        a = int(oracle.hash_bytes(width, seeds, data)[0])
        b = int(oracle.hash_bytes(width, seeds, other)[0])
        hits += (a & 0xFFFF) == (b & 0xFFFF)
    p = 2.0 ** (min(v, 16) - 16)
    mean, sd = trials * p, math.sqrt(trials * p * (1 - p))
    assert abs(hits - mean) <= 6 * sd + 1, (hits, mean, sd)
