"""Benchmark: HalftimeHash throughput on GB300 (one JSON line on stdout).

Default workload: one 1 GiB string of splitmix64(2) bytes, device-resident,
hashed at each output width (16, 24, 32, 40 bytes) under seed 7.  One step =
the four hashes (4 GiB hashed).  The input is larger than L2 (1 GiB vs
129 MB), so no flush is needed between launches.

  value   GB/s over the timed steps, CUDA events on the launching stream,
          max over ranks (each rank hashes its own copy: weak scaling).
  e2e     the same metric through ht_hash_host from pinned host memory: the
          host-to-device copy of every step's input and the digest read-back
          are inside the timed region.
  roofline  the dominant kernel (the slowest width) against the measured HBM
          copy bandwidth; algorithmic bytes = 2^30 read per launch.
  cpu_baseline  the CPU oracle on the host's cores: all cores at once
          (independent 64 MiB pieces of the string), one thread, and the
          whole string at every width (its digests checked against the GPU's).
  blocks_256  the same string and widths with 256-bit blocks (b = 4 words).
  tree_ablation  the same string and widths under the binary-tree ablation
          (Badger's approach) against the paper's tree.
  size_sweep  per-launch time of 1..256 MiB strings (widths 24, 40).
  batch   the 50,000-string batch: default and autotuned batch shape, the
          strings below one chunk and the rest, and one launch per string.

`--impl reference` times the CPU oracle instead (the reference arm): each step
hashes the whole string at each width, one oracle thread per width.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WIDTHS = (16, 24, 32, 40)
METRIC = "HalftimeHash GB/s hashed vs HBM roofline; served request p50/p99 latency"
SEED_DATA = 2
SEED_KEY = 7
GIB = 1 << 30


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _profiled_traffic(width, nbytes, shape):
    """DRAM bytes per launch from profiles/traffic.json, only while the kernel
    sources are those that were profiled and the launch is the profiled one
    (1 GiB, warp-chunk kernel with 64-execution chunks)."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        h = hashlib.sha256()
        for f in t["kernel_sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != t["kernel_sources_sha256"]:
            return None
        if nbytes != GIB or shape.get("kernel") != 1 or shape.get("chunk_levels") != 2:
            return None
        return t["bytes_per_launch"].get(str(width))
    except Exception:
        return None


def run_size_sweep(args):
    """Per-launch time of one width over string sizes 1 MiB .. 4 GiB (CUDA
    events, back-to-back launches): separates the fixed cost of a launch from
    the steady-state bandwidth."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2104_08865_gb300 import Hasher, abi, inputs
    dev = torch.device("cuda", 0)
    maxn = 4 * GIB
    data = inputs.stream_bytes_torch(SEED_DATA, 0, maxn, dev)
    out = torch.empty(5, dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream()
    rows = []
    for w in args.sweep_widths:
        h = Hasher(w, seed_words=abi.ht_seed_expand(SEED_KEY, w))
        for n in [1 << 20, 16 << 20, 64 << 20, 256 << 20, 512 << 20, GIB, 2 * GIB, 4 * GIB]:
            reps = max(5, min(200, (8 * GIB) // n))
            # successive launches read pieces at least 384 MiB apart (from HBM)
            copies = min(maxn // n, max(1, (384 << 20) // n + 1))
            at = [data.data_ptr() + (i % copies) * n for i in range(reps + 3)]
            for i in range(3):
                abi.ht_hash(h.ctx, at[i], n, out.data_ptr(), s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for i in range(reps):
                abi.ht_hash(h.ctx, at[3 + i], n, out.data_ptr(), s)
            e1.record(s)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1000 / reps
            rows.append({"width": w, "bytes": n, "us": round(us, 2), "gbs": round(n / us / 1e3, 1)})
        h.close()
    fits = {}
    for w in args.sweep_widths:
        a = [r for r in rows if r["width"] == w and r["bytes"] in (2 * GIB, 4 * GIB)]
        slope = (a[1]["us"] - a[0]["us"]) / (a[1]["bytes"] - a[0]["bytes"])  # us per byte
        fits[str(w)] = {"steady_gbs": round(1 / slope / 1e3, 1),
                        "fixed_us": round(a[1]["us"] - slope * a[1]["bytes"], 1)}
    print(json.dumps({"size_sweep": rows, "fit_2_to_4_gib": fits}), flush=True)
    return 0


def _oracle_gbs(data_np, n_bytes: int):
    """The oracle over the first n_bytes at every width, one thread per width."""
    import numpy as np

    import oracle
    sample = data_np[:n_bytes]
    seeds = {w: oracle.seed_expand(SEED_KEY, oracle.seed_words(w)) for w in WIDTHS}
    out = {}

    def run(w):
        out[w] = oracle.hash_bytes(w, seeds[w], sample)

    t0 = time.perf_counter()
    ths = [threading.Thread(target=run, args=(w,)) for w in WIDTHS]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    return len(WIDTHS) * n_bytes / dt / 1e9, dt, out


def _workload(nbytes: int) -> str:
    """The benchmark's workload, as both arms name it."""
    return ("one %d MiB string of splitmix64(%d) bytes, device-resident, hashed at widths "
            "16/24/32/40 (seed %d) per step" % (nbytes >> 20, SEED_DATA, SEED_KEY))


def _config(nbytes: int) -> dict:
    """The workload both arms name in `config`."""
    return {"workload": _workload(nbytes), "bytes_per_step": len(WIDTHS) * nbytes,
            "l2": "inputs larger than L2 (no flush)"}


def run_reference(args):
    """The reference arm: the CPU oracle on the same workload, the whole
    string at each of the four widths per step, one oracle thread per width
    (the oracle hashes one string serially)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2104_08865_gb300 import inputs
    nbytes = args.bytes
    data = inputs.stream_bytes(SEED_DATA, 0, nbytes)
    for _ in range(args.warmup):
        _oracle_gbs(data, nbytes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_gbs(data, nbytes)
    dt = time.perf_counter() - t0
    gbs = args.steps * len(WIDTHS) * nbytes / dt / 1e9
    desc = ("each step: the whole %d MiB string at each of the four widths, one oracle thread "
            "per width" % (nbytes >> 20))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * dt / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": _config(nbytes),
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": len(WIDTHS),
                         "host_cores": os.cpu_count(), "kind": "oracle", "sample": desc},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_threads_gbs(data_np, piece: int, threads: int):
    """`threads` oracle threads at once, thread i hashing its own piece of
    `piece` bytes of the string (pieces wrap around the string) at width
    WIDTHS[i % 4]: the host's throughput over independent strings."""
    import oracle
    seeds = {w: oracle.seed_expand(SEED_KEY, oracle.seed_words(w)) for w in WIDTHS}
    n = len(data_np)

    def run(i):
        o = (i * piece) % max(1, n - piece + 1)
        oracle.hash_bytes(WIDTHS[i % 4], seeds[WIDTHS[i % 4]], data_np[o:o + piece])

    t0 = time.perf_counter()
    ths = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    return threads * piece / dt / 1e9


def _aligned_offsets(lens, align=256):
    import numpy as np
    slots = (np.asarray(lens, dtype=np.int64) + align - 1) // align * align
    offs = np.concatenate([[0], np.cumsum(slots)[:-1]]).astype(np.int64)
    return offs, int(slots.sum())


def run_batch(args, dev, stream):
    """C4: 50,000 strings, lengths log-uniform in [64 B, 1 MiB] (splitmix64
    seed 3), width 24: one graph-replayed batch launch vs one launch per
    string.  String i occupies bytes [off_i, off_i + len_i) of the seed-3
    stream, with off_i 256-byte aligned."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, abi, inputs, shard
    ws, rank, _ = _dist()
    all_lens = inputs.log_uniform_lengths(3, args.batch_strings, 64, 1 << 20)
    # under torchrun each rank hashes a byte-balanced, contiguous share
    lo, hi = shard.shard_of(all_lens, ws, rank)
    lens = all_lens[lo:hi]
    count = len(lens)
    offs, total = _aligned_offsets(lens)
    buf = inputs.stream_bytes_torch(3, 0, total + 256, dev)
    ptrs = torch.tensor(buf.data_ptr() + offs, dtype=torch.int64, device=dev)
    lt = torch.tensor(lens, dtype=torch.int64, device=dev)
    h = Hasher(24, seed_words=abi.ht_seed_expand(SEED_KEY, 24))
    out = torch.empty((count, 3), dtype=torch.int64, device=dev)
    reps = 10

    def timed(p, l, n, o):
        for _ in range(3):
            abi.ht_hash_batch(h.ctx, p, l, n, o, stream)
        torch.cuda.synchronize()
        h.status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = h.launches()
        e0.record(stream)
        for _ in range(reps):
            abi.ht_hash_batch(h.ctx, p, l, n, o, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, (h.launches() - l0) // reps

    # the default batch shape, then the batch autotuner's pick (set-up, untimed)
    ms_default, _ = timed(ptrs, lt, count, out)
    default_shape = abi.ht_get_shape(h.ctx, 2**64 - 1)
    tuned_shape = abi.ht_autotune_batch(h.ctx, ptrs, lt, count, out, stream)
    ms_batch, launches_batch = timed(ptrs, lt, count, out)
    ms_batch = shard.max_over_ranks(ms_batch, dev)
    # strings below one 64-execution chunk and the rest, each as a batch
    chunk = 64 * 1344
    classes = {}
    for name, sel in (("under_one_chunk", lens < chunk), ("one_chunk_or_more", lens >= chunk)):
        idx = torch.tensor(np.nonzero(sel)[0], dtype=torch.int64, device=dev)
        m = int(idx.numel())
        if m == 0:
            continue
        o2 = torch.empty((m, 3), dtype=torch.int64, device=dev)
        ms_c, _ = timed(ptrs[idx].contiguous(), lt[idx].contiguous(), m, o2)
        b = int(lens[sel].sum())
        classes[name] = {"strings": m, "gb": round(b / 1e9, 3), "ms": round(ms_c, 3),
                         "gbs": round(b / ms_c / 1e6, 1)}
    nbytes = int(all_lens.sum())
    naive = torch.empty_like(out)
    hp = (buf.data_ptr() + offs).astype(np.uint64)
    h.hash_batch_naive(hp, lens, naive)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.hash_batch_naive(hp, lens, naive)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_naive = shard.max_over_ranks(e0.elapsed_time(e1), dev)
    same = bool(torch.equal(out, naive))
    h.close()
    return {"workload": "%d strings, log-uniform 64 B..1 MiB, %.2f GB, width 24%s" % (
                args.batch_strings, nbytes / 1e9, "" if ws == 1 else ", sharded by bytes over %d ranks" % ws),
            "batch_gbs": round(nbytes / ms_batch / 1e6, 1), "batch_ms": round(ms_batch, 3),
            "batch_launches": launches_batch, "tuned_shape": tuned_shape,
            "default_shape_gbs": round(nbytes / ms_default / 1e6, 1), "default_shape": default_shape,
            "classes": classes,
            "naive_gbs": round(nbytes / ms_naive / 1e6, 1), "naive_ms": round(ms_naive, 3),
            "naive_launches": args.batch_strings, "speedup": round(ms_naive / ms_batch, 2),
            "digests_equal": same}


def run_dedup(args, dev, stream):
    """Deduplication by content: the batch of 50,000 strings (log-uniform
    64 B .. 1 MiB, splitmix64 seed 3, width 24) plus 12,500 entries aliasing
    earlier strings' bytes, hashed in one batch launch and inserted into the
    digest table (representatives out).  Times the whole chain against the
    hashing alone; the representatives must be what the construction fixes
    (each original its own, each alias its original)."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, Table, abi, inputs
    lens = inputs.log_uniform_lengths(3, args.batch_strings, 64, 1 << 20)
    offs, total = _aligned_offsets(lens)
    buf = inputs.stream_bytes_torch(3, 0, total + 256, dev)
    rng = np.random.default_rng(8)
    alias = rng.integers(0, len(lens), len(lens) // 4)
    all_offs = np.concatenate([offs, offs[alias]])
    all_lens = np.concatenate([lens, lens[alias]])
    n = len(all_lens)
    ptrs = torch.tensor(buf.data_ptr() + all_offs, dtype=torch.int64, device=dev)
    lt = torch.tensor(all_lens, dtype=torch.int64, device=dev)
    h = Hasher(24, seed_words=abi.ht_seed_expand(SEED_KEY, 24))
    abi.ht_ctx_reserve(h.ctx, int(all_lens.sum()) + (1 << 20), n)
    dig = torch.empty((n, 3), dtype=torch.int64, device=dev)
    rep = torch.empty(n, dtype=torch.int32, device=dev)
    t = Table(h, max_entries=n, seed64=0x7AB1E)

    def chain():
        abi.ht_hash_batch(h.ctx, ptrs, lt, n, dig, stream)
        t.clear(stream)
        abi.ht_table_insert(t.t, dig, n, rep, stream)

    for _ in range(3):
        chain()
    torch.cuda.synchronize()
    t.status()
    got = rep.cpu().numpy().view(np.uint32).astype(np.int64)
    ok = bool(np.array_equal(got[:len(lens)], np.arange(len(lens))) and np.array_equal(got[len(lens):], alias))
    reps = 10
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(reps):
        abi.ht_hash_batch(h.ctx, ptrs, lt, n, dig, stream)
    e1.record(stream)
    for _ in range(reps):
        chain()
    e2.record(stream)
    torch.cuda.synchronize()
    ms_hash = e0.elapsed_time(e1) / reps
    ms_chain = e1.elapsed_time(e2) / reps
    nbytes = int(all_lens.sum())
    t.close()
    h.close()
    return {"workload": "%d strings (%d distinct, log-uniform 64 B..1 MiB), %.2f GB, width 24" % (
                n, len(lens), nbytes / 1e9),
            "chain_gbs": round(nbytes / ms_chain / 1e6, 1), "chain_ms": round(ms_chain, 3),
            "hash_only_ms": round(ms_hash, 3), "table_ms": round(ms_chain - ms_hash, 3),
            "distinct": int((got == np.arange(n)).sum()), "representatives_ok": ok}


def run_incremental(args, dev, stream, data, want):
    """The benchmark's string hashed incrementally at width 24 (init / update /
    final): device-resident pieces of 64 MiB and of 1 MiB + 3 bytes (every
    piece boundary inside a chunk, so each update also copies a partial
    chunk), both also with overlapping launches (HT_FLAG_OVERLAP_LAUNCHES),
    and pinned host pieces of 64 MiB through the host update.  The digest
    must equal the one-shot digest."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, abi
    w = 24
    n = data.numel()
    h = Hasher(w, seed_words=abi.ht_seed_expand(SEED_KEY, w))
    inc = h.incremental()
    out = torch.empty(w // 8, dtype=torch.int64, device=dev)
    res = {"workload": "one %d MiB string, width 24, fed in pieces" % (n >> 20)}

    def run_dev(piece):
        inc.init(stream)
        for o in range(0, n, piece):
            inc.update(data[o:o + piece], stream)
        inc.final(out, stream)

    same = True
    for name, piece, reps, flags in (("device_64mib", 64 << 20, 10, 0),
                                     ("device_1mib_plus_3", (1 << 20) + 3, 3, 0),
                                     ("device_64mib_overlapped", 64 << 20, 10, abi.HT_FLAG_OVERLAP_LAUNCHES),
                                     ("device_1mib_plus_3_overlapped", (1 << 20) + 3, 3,
                                      abi.HT_FLAG_OVERLAP_LAUNCHES)):
        abi.ht_ctx_set_flags(h.ctx, flags)
        run_dev(piece)
        torch.cuda.synchronize()
        same &= out.cpu().numpy().view(np.uint64).tolist() == want
        l0 = h.launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run_dev(piece)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"gbs": round(n / ms / 1e6, 1), "ms": round(ms, 3),
                     "launches": (h.launches() - l0) // reps}
    abi.ht_ctx_set_flags(h.ctx, 0)
    pinned = torch.empty(n, dtype=torch.uint8).pin_memory()
    pinned.copy_(data)
    hp = pinned.numpy()
    piece = 64 << 20

    def run_host():
        inc.init(stream)
        for o in range(0, n, piece):
            inc.update(hp[o:o + piece], stream)
        inc.final(out, stream)
        torch.cuda.synchronize()

    run_host()
    same &= out.cpu().numpy().view(np.uint64).tolist() == want
    t0 = time.perf_counter()
    for _ in range(3):
        run_host()
    dt = (time.perf_counter() - t0) / 3
    res["host_pinned_64mib"] = {"gbs": round(n / dt / 1e9, 1), "ms": round(dt * 1e3, 3)}
    res["digest_equals_one_shot"] = bool(same)
    inc.close()
    h.close()
    return res


def run_unaligned(args, stream, data, hashers, shapes, per_w):
    """The benchmark string 3 bytes past a 16-byte boundary (its bytes 3 ..
    n - 14, the same launch shape as the aligned string): each width timed
    alone as in the aligned per-launch figures."""
    import torch

    from paper_2104_08865_gb300 import abi
    nbytes = args.bytes
    off, n = 3, args.bytes - 16
    outs = {w: torch.empty(w // 8, dtype=torch.int64, device=data.device) for w in WIDTHS}
    for w in WIDTHS:
        sh = shapes[str(w)]
        abi.ht_set_shape(hashers[w].ctx, n, sh["kernel"], sh["chunk_levels"], sh["stages"],
                         sh["threads_per_block"], sh["blocks_per_sm"])

    def once(evs=None):
        for i, w in enumerate(WIDTHS):
            if evs is not None:
                evs[i][0].record(stream)
            abi.ht_hash(hashers[w].ctx, data.data_ptr() + off, n, outs[w].data_ptr(), stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(max(1, args.warmup)):
        once()
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in WIDTHS]
           for _ in range(5)]
    for ev in evs:
        once(ev)
    torch.cuda.synchronize()
    gbs = {}
    for i, w in enumerate(WIDTHS):
        ms = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for ev in evs)
        gbs[str(w)] = round(n / (ms / 1e3) / 1e9, 1)
    return {"offset": off, "bytes": n, "per_width_gbs": gbs,
            "vs_aligned": {str(w): round(gbs[str(w)] / (nbytes / (per_w[w] / 1e3) / 1e9), 3)
                           for w in WIDTHS}}


def run_v3(args, dev, stream, data):
    """The 256-bit-block variant (blocks of 4 words, width | HT_BLOCK_256) on the
    benchmark string: each width timed alone (CUDA events around each launch,
    default launch shape), then the four launches back to back with overlap,
    as in the main step."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, abi
    nbytes = args.bytes
    hs = {w: Hasher(w | abi.HT_BLOCK_256, seed_words=abi.ht_seed_expand(SEED_KEY, w | abi.HT_BLOCK_256))
          for w in WIDTHS}
    outs = {w: torch.empty(w // 8, dtype=torch.int64, device=dev) for w in WIDTHS}

    def step(evs=None):
        for i, w in enumerate(WIDTHS):
            if evs is not None:
                evs[i][0].record(stream)
            abi.ht_hash(hs[w].ctx, data.data_ptr(), nbytes, outs[w].data_ptr(), stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    reps = 30
    solo = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
             for _ in WIDTHS] for _ in range(reps)]
    for ev in solo:
        step(ev)
    torch.cuda.synchronize()
    per_w = {w: statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for ev in solo)
             for i, w in enumerate(WIDTHS)}
    for w in WIDTHS:
        abi.ht_ctx_set_flags(hs[w].ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
    for _ in range(3):
        step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peak, _ = _peaks()
    dom = max(WIDTHS, key=lambda w: per_w[w])
    res = {"workload": _workload(nbytes).replace("hashed at widths", "256-bit blocks, widths"),
           "step_gbs": round(len(WIDTHS) * nbytes / ms / 1e6, 1), "ms_per_step": round(ms, 4),
           "per_width_gbs": {str(w): round(nbytes / per_w[w] / 1e6, 1) for w in WIDTHS},
           "dominant_frac_of_peak": round(nbytes / per_w[dom] / 1e6 / peak, 4),
           "shape": abi.ht_get_shape(hs[dom].ctx, nbytes),
           "digests": {str(w): ["%016x" % v for v in outs[w].cpu().numpy().view(np.uint64)] for w in WIDTHS}}
    for h in hs.values():
        h.close()
    return res


def run_tree_ablation(args, dev, stream, data):
    """The binary-tree ablation (width | HT_TREE_BINARY: Badger's approach,
    Eq. algebraic-badger over all EHC outputs, no final NH) against the
    paper's tree on the benchmark string: each width's launch timed alone
    with CUDA events, default launch shapes, both trees."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, abi
    nbytes = args.bytes
    res = {"workload": _workload(nbytes).replace("hashed at widths", "tree T-hat vs binary tree, widths"),
           "per_width": {}}
    reps = 20
    for w in WIDTHS:
        row = {}
        for name, code in (("t_hat", w), ("binary", w | abi.HT_TREE_BINARY)):
            h = Hasher(code, seed_words=abi.ht_seed_expand(SEED_KEY, code))
            out = torch.empty(w // 8, dtype=torch.int64, device=dev)
            for _ in range(3):
                abi.ht_hash(h.ctx, data.data_ptr(), nbytes, out.data_ptr(), stream)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, b in evs:
                a.record(stream)
                abi.ht_hash(h.ctx, data.data_ptr(), nbytes, out.data_ptr(), stream)
                b.record(stream)
            torch.cuda.synchronize()
            h.status()
            us = statistics.mean(a.elapsed_time(b) for a, b in evs) * 1000
            row[name] = {"us": round(us, 2), "gbs": round(nbytes / us / 1e3, 1),
                         "digest": ["%016x" % v for v in out.cpu().numpy().view(np.uint64)]}
            h.close()
        row["binary_over_t_hat_time"] = round(row["binary"]["us"] / row["t_hat"]["us"], 3)
        res["per_width"][str(w)] = row
    return res


def run_size_sweep_leg(args, dev, stream, data):
    """Per-launch time of single strings of 1 to 256 MiB (widths 24 and 40,
    the default launch shape of each length): back-to-back launches timed
    with CUDA events (the fixed cost of a launch against its bytes), and the
    median of 20 lone launches (events around one launch, synchronised).
    Successive launches hash successive n-byte pieces of the 1 GiB string,
    at least 384 MiB apart before one is read again, so every launch reads
    from HBM, not from the L2 cache."""
    import torch

    from paper_2104_08865_gb300 import Hasher, abi
    rows = []
    for w in (24, 40):
        h = Hasher(w, seed_words=abi.ht_seed_expand(SEED_KEY, w))
        out = torch.empty(w // 8, dtype=torch.int64, device=dev)
        for mib in (1, 4, 16, 64, 256):
            n = mib << 20
            copies = min(data.numel() // n, max(1, (384 << 20) // n + 1))
            at = [data.data_ptr() + (i % copies) * n for i in range(400)]
            for i in range(3):
                abi.ht_hash(h.ctx, at[i], n, out.data_ptr(), stream)
            reps = max(10, min(200, (2 * GIB) // n))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(reps):
                abi.ht_hash(h.ctx, at[i], n, out.data_ptr(), stream)
            e1.record(stream)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1000 / reps
            lone = []
            for i in range(20):
                e0.record(stream)
                abi.ht_hash(h.ctx, at[200 + i], n, out.data_ptr(), stream)
                e1.record(stream)
                torch.cuda.synchronize()
                lone.append(e0.elapsed_time(e1) * 1000)
            # the same back to back with HT_FLAG_OVERLAP_LAUNCHES (each launch
            # may start while the one before it drains)
            abi.ht_ctx_set_flags(h.ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
            for i in range(3):
                abi.ht_hash(h.ctx, at[i], n, out.data_ptr(), stream)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(reps):
                abi.ht_hash(h.ctx, at[i], n, out.data_ptr(), stream)
            e1.record(stream)
            torch.cuda.synchronize()
            us_ov = e0.elapsed_time(e1) * 1000 / reps
            abi.ht_ctx_set_flags(h.ctx, 0)
            shape = abi.ht_get_shape(h.ctx, n)
            rows.append({"width": w, "mib": mib, "us": round(us, 2), "gbs": round(n / us / 1e3, 1),
                         "overlapped_us": round(us_ov, 2), "overlapped_gbs": round(n / us_ov / 1e3, 1),
                         "lone_us": round(statistics.median(lone), 2),
                         "kernel": {1: "warp-chunk", 3: "block-chunk"}.get(shape["kernel"], shape["kernel"]),
                         "chunk_levels": shape["chunk_levels"]})
        h.status()
        h.close()
    return {"note": "per-launch time, default shape per length, cold pieces; us = back-to-back mean, "
                    "overlapped_us = the same with HT_FLAG_OVERLAP_LAUNCHES, "
                    "lone_us = median of one launch between events", "rows": rows}


def run_serving(args, dev, stream):
    """C5: Poisson arrivals of width-32 hash requests, lengths log-uniform in
    [256 B, 64 MiB], 16 GiB admission budget; offered load swept over
    fractions of the peak measured for each form (device-resident requests,
    and pinned host requests copied in by the server)."""
    import numpy as np
    import torch

    from paper_2104_08865_gb300 import Hasher, abi, inputs
    rng = np.random.default_rng(6)
    pool_bytes = args.serve_pool
    pool_dev = inputs.stream_bytes_torch(5, 0, pool_bytes, dev)
    pool_host = torch.empty(pool_bytes, dtype=torch.uint8).pin_memory()
    pool_host.copy_(pool_dev)
    torch.cuda.synchronize()
    h = Hasher(32, seed_words=abi.ht_seed_expand(SEED_KEY, 32))
    mean_len = None
    out = {"workload": "width 32, lengths log-uniform 256 B..64 MiB, Poisson arrivals, budget 16 GiB, "
                       "8 batches in flight, %.1f s per load point" % args.serve_seconds, "forms": {},
           "form_notes": {"device": "requests already in device memory",
                          "pinned_h2d": "pinned host requests read in place by the batch kernel over "
                                        "the CPU-GPU link (the server's default)",
                          "pinned_h2d_staged": "pinned host requests copied into a device arena first"}}

    def requests(n, seed):
        ln = inputs.log_uniform_lengths(seed, n, 256, 64 << 20)
        off = (rng.integers(0, pool_bytes - (64 << 20), n) // 256) * 256
        return ln, off

    # pinned host requests: read in place by the batch kernel over the
    # CPU-GPU link (the server's default), and staged through device memory
    for form, base, pinned, mode in (("device", pool_dev.data_ptr(), 0, 0),
                                     ("pinned_h2d", pool_host.data_ptr(), 1, 0),
                                     ("pinned_h2d_staged", pool_host.data_ptr(), 1, 1)):
        res = {}
        # peak: bursts with every request arriving at once, sized to tens of
        # milliseconds of work; the better of two
        nburst = 10000 if form == "device" else 2000
        ln, off = requests(nburst, 61)
        srv = abi.ht_server_create(h.ctx, 16 << 30, n_streams=8, max_batch=4096, pinned_mode=mode)
        dig = np.zeros((nburst, 4), dtype=np.uint64)
        peak = 0.0
        for _ in range(2):
            abi.ht_server_replay(srv, base + off, ln, [pinned] * nburst, np.zeros(nburst), dig)
            st = abi.ht_server_stats(srv, reset=True)
            gbs = st["bytes_completed"] / st["wall_s"] / 1e9
            if gbs > peak:
                peak, peak_batches = gbs, st["batches"]
        res["peak_gbs"] = round(peak, 1)
        res["peak_batches"] = int(peak_batches)
        mean_len = float(inputs.log_uniform_lengths(62, 100000, 256, 64 << 20).mean())
        res["points"] = []
        for frac in args.serve_loads:
            rate = frac * peak * 1e9 / mean_len  # requests per second
            n = max(50, int(rate * args.serve_seconds))
            # device-resident requests below saturation: several runs of the
            # point (fresh arrivals each), the median run reported with the
            # spread of p50 and p99
            runs = args.serve_repeats if (form == "device" and frac < 1) else 1
            sts = []
            for _ in range(runs):
                ln, off = requests(n, 63)
                gaps = rng.exponential(1e6 / rate, n)
                arr = np.cumsum(gaps) - gaps[0]
                dig = np.zeros((n, 4), dtype=np.uint64)
                late = abi.ht_server_replay(srv, base + off, ln, [pinned] * n, arr, dig)
                st = abi.ht_server_stats(srv, reset=True)
                st["late"] = late
                sts.append(st)
            sts.sort(key=lambda v: v["p99_us"])
            st = sts[len(sts) // 2]
            pt = {"load": frac, "offered_gbs": round(frac * peak, 1),
                  "requests": n, "achieved_gbs": round(st["bytes_completed"] / st["wall_s"] / 1e9, 1),
                  "p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1),
                  "max_submit_delay_us": round(st["late"], 1), "batches": int(st["batches"])}
            if runs > 1:
                pt["runs"] = runs
                pt["p50_us_range"] = [round(min(v["p50_us"] for v in sts), 1), round(max(v["p50_us"] for v in sts), 1)]
                pt["p99_us_range"] = [round(sts[0]["p99_us"], 1), round(sts[-1]["p99_us"], 1)]
            res["points"].append(pt)
        abi.ht_server_destroy(srv)
        out["forms"][form] = res
    out["mean_len_bytes"] = round(mean_len)
    h.close()
    del pool_host
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import __graft_entry__
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2104_08865_gb300", "libhalftime.so")):
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_2104_08865_gb300 import Hasher, abi, inputs

    nbytes = args.bytes
    stream = torch.cuda.current_stream()
    data = inputs.stream_bytes_torch(SEED_DATA, 0, nbytes, dev)
    hashers = {w: Hasher(w, seed_words=abi.ht_seed_expand(SEED_KEY, w)) for w in WIDTHS}
    shapes = {}
    for w in WIDTHS:
        if args.shape:
            kern, L, st, tpb, bps = (int(v) for v in args.shape.split(","))
            abi.ht_set_shape(hashers[w].ctx, nbytes, kern, L, st, tpb, bps)
        elif not args.no_autotune:
            abi.ht_autotune(hashers[w].ctx, nbytes, stream)
        shapes[str(w)] = abi.ht_get_shape(hashers[w].ctx, nbytes)
    outs = {w: torch.empty(w // 8, dtype=torch.int64, device=dev) for w in WIDTHS}

    def step(evs=None):
        for i, w in enumerate(WIDTHS):
            if evs is not None:
                evs[i][0].record(stream)
            abi.ht_hash(hashers[w].ctx, data.data_ptr(), nbytes, outs[w].data_ptr(), stream)
            if evs is not None:
                evs[i][1].record(stream)

    # per-launch times for the roofline: each launch alone, bracketed by events
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    solo = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
             for _ in WIDTHS] for _ in range(max(3, min(args.steps, 50)))]
    for ev in solo:
        step(ev)
    torch.cuda.synchronize()
    per_w = {}
    for i, w in enumerate(WIDTHS):
        per_w[w] = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for ev in solo)
    unaligned = run_unaligned(args, stream, data, hashers, shapes, per_w) if rank == 0 else None
    # the timed step: the four launches back to back; with overlap on, each
    # launch may start while the previous one drains (its input is never the
    # previous launch's output)
    if not args.no_overlap:
        for w in WIDTHS:
            abi.ht_ctx_set_flags(hashers[w].ctx, abi.HT_FLAG_OVERLAP_LAUNCHES)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches0 = sum(h.launches() for h in hashers.values())
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for s in range(args.steps):
        step()
    t_end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    launches = sum(h.launches() for h in hashers.values()) - launches0
    ms_total = t_start.elapsed_time(t_end)
    if ws > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    total_bytes = ws * args.steps * len(WIDTHS) * nbytes
    value = total_bytes / (ms_total / 1e3) / 1e9
    dom = max(WIDTHS, key=lambda w: per_w[w])
    peak, peak_kind = _peaks()
    achieved = nbytes / (per_w[dom] / 1e3) / 1e9
    traffic = _profiled_traffic(dom, nbytes, shapes.get(str(dom), {}))
    digests = {w: outs[w].cpu().numpy().view(np.uint64).tolist() for w in WIDTHS}

    # ---- end to end: pinned host input through ht_hash_host ---------------
    e2e = None
    if not args.no_e2e:
        host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        host.copy_(data)
        hnp = host.numpy()
        dig = np.zeros(5, dtype=np.uint64)
        for w in WIDTHS:  # warm-up (staging ring allocation)
            abi.ht_hash_host(hashers[w].ctx, hnp.ctypes.data, nbytes, dig.ctypes.data, stream)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(e_steps):
            for w in WIDTHS:
                abi.ht_hash_host(hashers[w].ctx, hnp.ctypes.data, nbytes, dig.ctypes.data, stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": round(ws * e_steps * len(WIDTHS) * nbytes / dt / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": len(WIDTHS) * nbytes,
               "d2h_bytes_per_step": sum(w for w in WIDTHS), "steps": e_steps,
               "path": "ht_hash_host: pinned host -> device in 64 MiB pieces overlapped with hashing"}
        del host

    # ---- CPU oracle baseline (rank 0, N = 1 only) --------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        host_np = data.cpu().numpy()
        sample = min(nbytes, args.cpu_bytes)
        # the whole string at every width, one thread per width: the digests
        # must equal the GPU's
        gbs4, dt, ref = _oracle_gbs(host_np, sample)
        match = None
        if sample == nbytes:
            match = all(np.array_equal(np.asarray(digests[w], dtype=np.uint64), ref[w]) for w in WIDTHS)
        cores = os.cpu_count() or 1
        piece = min(64 << 20, nbytes)
        single = _oracle_threads_gbs(host_np, piece, 1)
        allc = _oracle_threads_gbs(host_np, piece, cores)
        cpu = {"value": round(allc, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
               "host_cores": cores,
               "sample": "all host cores: %d oracle threads at once, each hashing its own %d MiB piece "
                         "of the string (widths in turn)" % (cores, piece >> 20),
               "single_thread_gbs": round(single, 4),
               "single_thread_sample": "one oracle thread, a %d MiB piece at width 16" % (piece >> 20),
               "four_widths_gbs": round(gbs4, 4),
               "four_widths_sample": "the whole %d MiB string at each width, one thread per width "
                                     "(%.1f s)" % (sample >> 20, dt),
               "digests_match_gpu": match}

    v3 = run_v3(args, dev, stream, data) if (rank == 0 and not args.no_v3) else None
    ablation = run_tree_ablation(args, dev, stream, data) if (rank == 0 and not args.no_ablation) else None
    sweep = run_size_sweep_leg(args, dev, stream, data) if (rank == 0 and not args.no_sweep) else None
    batch = run_batch(args, dev, stream) if not args.no_batch else None
    incremental = (run_incremental(args, dev, stream, data, digests[24])
                   if (rank == 0 and not args.no_inc) else None)
    dedup = run_dedup(args, dev, stream) if (rank == 0 and not args.no_dedup) else None
    serving = run_serving(args, dev, stream) if (rank == 0 and not args.no_serve) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": _config(nbytes),
            "timing": {"launches": "back to back on one stream" + (
                           "" if args.no_overlap else ", overlapping (programmatic dependent launch)"),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "per_width_gbs": {str(w): round(nbytes / (per_w[w] / 1e3) / 1e9, 2) for w in WIDTHS},
            "per_width_note": "each launch alone, bracketed by CUDA events (no overlap)",
            "unaligned": unaligned,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": "%s<%d> (single string)" % (
                             "stream_kernel" if shapes[str(dom)]["kernel"] == 0 else "hash_kernel", dom),
                         "peak_source": peak_kind},
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": ck,
            "shapes": shapes,
            "batch": batch, "incremental": incremental, "dedup": dedup, "serving": serving,
            "blocks_256": v3, "tree_ablation": ablation, "size_sweep": sweep,
            "digests": {str(w): ["%016x" % v for v in digests[w]] for w in WIDTHS},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bytes", type=int, default=GIB, help="string size (profiling runs use less)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape instead of autotuning it (setup, untimed)")
    ap.add_argument("--shape", default="", help="force a launch shape kernel,chunk_levels,stages,threads_per_block,blocks_per_sm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-bytes", type=int, default=GIB)
    ap.add_argument("--size-sweep", action="store_true",
                    help="print per-launch times over string sizes instead of the benchmark line")
    ap.add_argument("--sweep-widths", type=lambda v: [int(x) for x in v.split(",")], default=[24, 40])
    ap.add_argument("--no-overlap", action="store_true",
                    help="time the step without overlapping consecutive launches")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-inc", action="store_true", help="skip the incremental-hashing leg")
    ap.add_argument("--no-dedup", action="store_true", help="skip the deduplication leg")
    ap.add_argument("--no-v3", action="store_true", help="skip the 256-bit-block leg")
    ap.add_argument("--no-ablation", action="store_true", help="skip the binary-tree ablation leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-size launch-time leg")
    ap.add_argument("--batch-strings", type=int, default=50_000)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-repeats", type=int, default=3,
                    help="runs of each device-form load point below saturation")
    ap.add_argument("--serve-pool", type=int, default=2 * GIB)
    ap.add_argument("--serve-loads", type=lambda v: [float(x) for x in v.split(",")],
                    default=[0.1, 0.5, 0.9, 1.2])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and args.steps > 2:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.size_sweep:
        return run_size_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
