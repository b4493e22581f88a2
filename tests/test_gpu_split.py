"""One string hashed in parts and the parts' states combined (the split path
of a long string across devices): the digest equals the whole-string digest
and the oracle's, bit for bit."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2104_08865_gb300 import inputs, shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(built):
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _hasher(width, seed=7):
    from paper_2104_08865_gb300 import Hasher, abi
    return Hasher(width, seed_words=abi.ht_seed_expand(seed, width))


@pytest.mark.parametrize("width", [16, 24, 32, 40])
def test_parts_merged_on_one_gpu(dev, width):
    from paper_2104_08865_gb300 import abi
    xb = oracle.params(width)["exec_bytes"]
    gran = 64 * xb
    ref = oracle.seed_expand(7, oracle.seed_words(width))
    cases = [
        # (total length, split points as multiples of the granule)
        (3 * 512 * 64 * xb + 5 * 64 * xb + 3 * xb + 99, [700, 1100]),   # splits inside level-3 and -4 groups
        (8 * 512 * 64 * xb, [8 * 512 // 2]),                            # exact tree, even halves
        (50 * gran + 7 * xb + 5, [50]),                                 # last part = partial chunk + tail
        (gran - 1, []),                                                 # one part, shorter than a granule
        (0, []),
    ]
    total_max = max(c[0] for c in cases)
    data = inputs.stream_bytes_torch(17, 0, total_max + 16, dev)
    whole = _hasher(width)
    parts = [_hasher(width) for _ in range(3)]
    host = data.cpu().numpy()
    for total, cuts in cases:
        bounds = [0] + [c * gran for c in cuts] + [total]
        for h in parts:
            abi.ht_part_begin(h.ctx, total)
        for i in range(len(bounds) - 1):
            lo, hi = bounds[i], bounds[i + 1]
            abi.ht_hash_part(parts[i].ctx, data.data_ptr() + lo, lo, hi - lo)
        for i in range(1, len(bounds) - 1):
            ptr, words = abi.ht_part_state(parts[i].ctx)
            abi.ht_part_merge(parts[0].ctx, ptr, words)
        got = torch.empty(width // 8, dtype=torch.int64, device=dev)
        abi.ht_finish_parts(parts[0].ctx, got.data_ptr())
        want = whole.hash(data, total)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (width, total, cuts)
        assert np.array_equal(got.cpu().numpy().view(np.uint64), oracle.hash_bytes(width, ref, host[:total]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _split_rank(rank, world, port, out_dir, total):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cuda:0")
        data = inputs.stream_bytes_torch(18, 0, total, dev)
        h = _hasher(32)
        digest = shard.hash_split(h, data, total, world, rank)
        np.save(os.path.join(out_dir, "split%d.npy" % rank), digest)
    finally:
        dist.destroy_process_group()


def test_split_across_two_gloo_ranks(dev, tmp_path):
    """Two processes (ranks) on the one GPU of this machine each hash half of a
    string; a gloo all-reduce sums their states; both finish the digest of
    the whole string.  The ranks' kernels never wait on one another."""
    import torch.multiprocessing as mp
    total = (300 << 20) + 12345
    mp.start_processes(_split_rank, args=(2, _free_port(), str(tmp_path), total), nprocs=2,
                       start_method="spawn", join=True)
    data = inputs.stream_bytes_torch(18, 0, total, dev)
    want = _hasher(32).hash(data).cpu().numpy().view(np.uint64)
    for r in range(2):
        assert np.array_equal(np.load(str(tmp_path / ("split%d.npy" % r))), want)
