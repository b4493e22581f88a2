"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every entry point the headers declare, the host seed expansion
agrees with the oracle's, argument errors are reported, and the serving
loop's host logic behaves (through the host-only fake server)."""
import ctypes
import glob
import os
import re
import threading
import time

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ht_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(built):
    from paper_2104_08865_gb300 import abi
    declared = _header_functions()
    assert "ht_hash" in declared and "ht_server_submit" in declared
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    # the binding covers the same names
    assert set(abi.exported_symbols()) == declared


def test_checked_build_exports_the_same_symbols(built):
    """libhalftime_check.so (range-checked kernels) has every entry point and
    says it is the checked build; the product library says it is not."""
    from paper_2104_08865_gb300 import abi
    lib = ctypes.CDLL(os.path.join(os.path.dirname(abi.LIB_PATH), "libhalftime_check.so"))
    for name in sorted(_header_functions()):
        assert hasattr(lib, name), name
    lib.ht_build_flags.restype = ctypes.c_uint
    assert lib.ht_build_flags() == abi.HT_BUILD_CHECKED
    assert abi.ht_build_flags() == 0


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_seed_expansion_matches_oracle(built, width):
    from paper_2104_08865_gb300 import abi
    assert abi.ht_seed_words(width) == oracle.seed_words(width)
    for s in (0, 7, 2**64 - 1):
        assert np.array_equal(abi.ht_seed_expand(s, width), oracle.seed_expand(s, oracle.seed_words(width)))


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_seed_expansion_256_bit_blocks_matches_oracle(built, width):
    from paper_2104_08865_gb300 import abi
    code = width | abi.HT_BLOCK_256
    assert abi.ht_seed_words(code) == oracle.seed_words(width, 4)
    assert np.array_equal(abi.ht_seed_expand(7, code), oracle.seed_expand(7, oracle.seed_words(width, 4)))


def test_256_bit_blocks_rejected_where_unsupported(built):
    """The allocation-free call takes 8-word blocks only; it refuses the
    256-bit-block code before any CUDA work.  Unknown flag bits are refused."""
    from paper_2104_08865_gb300 import abi
    code = 24 | abi.HT_BLOCK_256
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_hash_noalloc(code, abi.ht_seed_expand(7, code), 0, 0, 0)
    assert e.value.code == abi.HT_ERR_WIDTH
    assert abi.ht_seed_words(24 | 0x400) == 0
    assert abi.ht_seed_words(abi.HT_BLOCK_256) == 0
    assert abi.ht_seed_words(24 | abi.HT_BLOCK_256 | abi.HT_TREE_BINARY) == 0
    assert abi.ht_seed_words(abi.HT_TREE_BINARY) == 0


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_seed_expansion_binary_tree_matches_oracle(built, width):
    """The binary-tree ablation's seed layout (E, 64 level keys per output
    word, R) has the oracle's size and words; the allocation-free call
    refuses the ablation before any CUDA work."""
    from paper_2104_08865_gb300 import abi
    code = width | abi.HT_TREE_BINARY
    assert abi.ht_seed_words(code) == oracle.seed_words_badger(width)
    assert np.array_equal(abi.ht_seed_expand(7, code), oracle.seed_expand(7, oracle.seed_words_badger(width)))
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_hash_noalloc(code, abi.ht_seed_expand(7, code), 0, 0, 0)
    assert e.value.code == abi.HT_ERR_WIDTH


def test_argument_errors(built):
    from paper_2104_08865_gb300 import abi
    assert abi.ht_seed_words(17) == 0
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_seed_expand(1, 17)
    assert e.value.code == abi.HT_ERR_WIDTH
    out = np.zeros(10, dtype=np.uint64)
    rc = abi.lib().ht_seed_expand(1, 24, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 10)
    assert rc == abi.HT_ERR_ARG
    code, msg = abi.ht_last_error()
    assert code == abi.HT_ERR_ARG and "4245" in msg
    with pytest.raises(abi.HalftimeError) as e:
        abi.ht_ctx_create(24, np.zeros(3, dtype=np.uint64))
    assert e.value.code == abi.HT_ERR_ARG


# ---------------------------------------------------------------- fake server

def test_fake_server_completes_and_reports_latency(built):
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(32, 1 << 20, batch_delay_us=2000, n_streams=2, max_batch=8)
    try:
        digs = np.ones((20, 4), dtype=np.uint64)
        tickets = [abi.ht_server_submit(srv, 0x1000 + i, 1000, False, digs[i:i + 1]) for i in range(20)]
        for t in tickets:
            abi.ht_server_wait(srv, t, 5_000_000)
            assert abi.ht_server_poll(srv, t)
        assert not digs.any()  # fake digests are zeros
        st = abi.ht_server_stats(srv)
        assert st["completed"] == 20 and st["batches"] >= 3  # max_batch 8
        assert st["p50_us"] >= 1500 and st["p99_us"] >= st["p50_us"]
        assert len(abi.ht_server_latencies(srv, 100)) == 20
    finally:
        abi.ht_server_destroy(srv)


def test_fake_server_budget_admission(built):
    """Requests wait for budget: with room for one 600-byte request at a time,
    three of them run in three batches, one after another."""
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(16, 1000, batch_delay_us=20000, n_streams=4)
    try:
        digs = np.zeros((3, 2), dtype=np.uint64)
        t0 = time.time()
        ts = [abi.ht_server_submit(srv, 0x1000, 600, True, digs[i:i + 1]) for i in range(3)]
        for t in ts:
            abi.ht_server_wait(srv, t, 5_000_000)
        assert time.time() - t0 >= 0.055
        assert abi.ht_server_stats(srv)["batches"] == 3
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_submit(srv, 0x1000, 1001, False, digs[:1])
        assert e.value.code == abi.HT_ERR_BUDGET
        assert abi.ht_server_stats(srv)["rejected"] == 1
    finally:
        abi.ht_server_destroy(srv)


def test_fake_server_timeout_cancel_and_queue_limit(built):
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(24, 100, batch_delay_us=300000, n_streams=1, max_queue=2)
    try:
        d = np.zeros((4, 3), dtype=np.uint64)
        a = abi.ht_server_submit(srv, 0x1000, 100, False, d[0:1])  # fills the budget
        time.sleep(0.02)
        b = abi.ht_server_submit(srv, 0x1000, 50, False, d[1:2])   # queued behind it
        c = abi.ht_server_submit(srv, 0x1000, 50, False, d[2:3])
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_submit(srv, 0x1000, 50, False, d[3:4])
        assert e.value.code == abi.HT_ERR_BUSY
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_wait(srv, a, 1000)  # bounded wait runs out
        assert e.value.code == abi.HT_ERR_TIMEOUT
        abi.ht_server_cancel(srv, c)
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_wait(srv, c, 1000)
        assert e.value.code == abi.HT_ERR_ARG
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_cancel(srv, a)  # already launched
        assert e.value.code == abi.HT_ERR_BUSY
        abi.ht_server_wait(srv, a, 5_000_000)
        abi.ht_server_wait(srv, b, 5_000_000)
        abi.ht_server_drain(srv, 5_000_000)
    finally:
        abi.ht_server_destroy(srv)


def test_fake_server_injected_failure_propagates(built):
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(40, 1 << 20, batch_delay_us=1000, fail_batch=1, n_streams=1,
                                    max_batch=1)
    try:
        d = np.zeros((3, 5), dtype=np.uint64)
        ts = [abi.ht_server_submit(srv, 0x1000, 10, False, d[i:i + 1]) for i in range(3)]
        abi.ht_server_wait(srv, ts[0], 5_000_000)
        with pytest.raises(abi.HalftimeError) as e:
            abi.ht_server_wait(srv, ts[1], 5_000_000)
        assert e.value.code == abi.HT_ERR_CUDA
        abi.ht_server_wait(srv, ts[2], 5_000_000)  # the server keeps serving
    finally:
        abi.ht_server_destroy(srv)


def test_fake_server_concurrent_submitters(built):
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(16, 1 << 16, batch_delay_us=500, n_streams=3, max_batch=16)
    try:
        d = np.zeros((400, 2), dtype=np.uint64)
        tickets = [None] * 400

        def worker(lo):
            for i in range(lo, lo + 100):
                tickets[i] = abi.ht_server_submit(srv, 0x1000, 64 + i, False, d[i:i + 1])

        ths = [threading.Thread(target=worker, args=(i * 100,)) for i in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        abi.ht_server_drain(srv, 10_000_000)
        assert all(abi.ht_server_poll(srv, t) for t in tickets)
        st = abi.ht_server_stats(srv)
        assert st["completed"] == 400
        assert st["bytes_completed"] == sum(64 + i for i in range(400))
    finally:
        abi.ht_server_destroy(srv)


def test_fake_server_replay_follows_arrival_times(built):
    from paper_2104_08865_gb300 import abi
    srv = abi.ht_server_create_fake(24, 1 << 30, batch_delay_us=200, n_streams=4, max_batch=64)
    try:
        n = 300
        arrivals = np.linspace(0, 30_000, n)  # 30 ms
        digs = np.ones((n, 3), dtype=np.uint64)
        t0 = time.time()
        late = abi.ht_server_replay(srv, [0x1000] * n, [4096] * n, None, arrivals, digs)
        assert time.time() - t0 >= 0.03
        assert late < 20_000
        assert not digs.any()
        st = abi.ht_server_stats(srv)
        assert st["completed"] == n and st["p99_us"] >= 200
    finally:
        abi.ht_server_destroy(srv)
