"""The N > 1 path on CPU: two gloo ranks shard a batch by bytes, each hashes
its strings (the oracle stands in for the GPU here), the digests are
gathered and the max-over-ranks timing helper agrees on every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_08865_gb300 import inputs, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        width = 24
        lens = inputs.log_uniform_lengths(3, 300, 64, 64 << 10)
        buf, offs = inputs.packed_batch(3, lens)
        seeds = oracle.seed_expand(7, oracle.seed_words(width))
        lo, hi = shard.shard_of(lens, world, rank)
        local = oracle.hash_many(width, seeds, buf, offs[lo:hi], lens[lo:hi])
        b = shard.shard_bounds(lens, world)
        counts = [int(b[r + 1] - b[r]) for r in range(world)]
        full = shard.gather_digests(local, counts)
        worst = shard.max_over_ranks(float(rank + 1))
        np.save(os.path.join(out_dir, "rank%d.npy" % rank), full)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%g" % worst)
    finally:
        dist.destroy_process_group()


def test_shard_bounds_balance_bytes():
    lens = inputs.log_uniform_lengths(3, 5000, 64, 1 << 20)
    for world in (1, 2, 3, 8):
        b = shard.shard_bounds(lens, world)
        assert b[0] == 0 and b[-1] == len(lens) and np.all(np.diff(b) >= 0)
        per = [int(lens[b[r]:b[r + 1]].sum()) for r in range(world)]
        assert sum(per) == int(lens.sum())
        assert max(per) - min(per) <= 2 * int(lens.max())
    assert list(shard.shard_bounds([0, 0, 0, 0], 2)) == [0, 2, 4]


def test_two_gloo_ranks_shard_and_gather(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    width = 24
    lens = inputs.log_uniform_lengths(3, 300, 64, 64 << 10)
    buf, offs = inputs.packed_batch(3, lens)
    seeds = oracle.seed_expand(7, oracle.seed_words(width))
    want = oracle.hash_many(width, seeds, buf, offs, lens)
    for r in range(world):
        got = np.load(str(tmp_path / ("rank%d.npy" % r)))
        assert np.array_equal(got, want)
        assert float(open(str(tmp_path / ("rank%d.txt" % r))).read()) == world
