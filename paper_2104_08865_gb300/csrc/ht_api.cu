// ht_api.cu -- host runtime of libhalftime: seeds, contexts, single-string,
// host-pipelined, batched (graph-replayed) and one-launch-per-string hashing,
// launch shapes and the autotuner.  See include/halftime.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "halftime.h"
#include "halftime_testing.h"
#include "ht_internal.h"
#include "ht_check.cuh"
#include "ht_runtime.h"
#include "ht_spec.cuh"

namespace ht {

// One range check of the checked build on (index, limit), touching nothing at
// index (a test of the recorder).
__global__ void check_probe_kernel(Ctl *ctl, uint64_t index, uint64_t limit) {
#ifdef HT_CHECK
  KParams P;
  P.scr.ctl = ctl;
  (void)HT_IN_RANGE(P, kChkInput, index, limit);
#else
  (void)ctl;
  (void)index;
  (void)limit;
#endif
}

// ---- errors ---------------------------------------------------------------------

static thread_local int g_err_code = HT_OK;
static thread_local char g_err_msg[256] = "";

int set_error(int code, const char *fmt, ...) {
  g_err_code = code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err_msg, sizeof g_err_msg, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  return set_error(e == cudaErrorMemoryAllocation ? HT_ERR_NOMEM : HT_ERR_CUDA,
                   "%s: %s", what, cudaGetErrorString(e));
}

#define HT_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_error(e_, #call); \
  } while (0)

const KernelSet *kernel_set(int width) {
  switch (width) {
    case 16: return &kernels_w16();
    case 24: return &kernels_w24();
    case 32: return &kernels_w32();
    case 40: return &kernels_w40();
    case 16 | HT_BLOCK_256: return &kernels_w16_v3();
    case 24 | HT_BLOCK_256: return &kernels_w24_v3();
    case 32 | HT_BLOCK_256: return &kernels_w32_v3();
    case 40 | HT_BLOCK_256: return &kernels_w40_v3();
    case 16 | HT_TREE_BINARY: return &kernels_w16_bin();
    case 24 | HT_TREE_BINARY: return &kernels_w24_bin();
    case 32 | HT_TREE_BINARY: return &kernels_w32_bin();
    case 40 | HT_TREE_BINARY: return &kernels_w40_bin();
    default: return nullptr;
  }
}

// ---- seeds: splitmix64 (Steele, Lea, Flood 2014) ------------------------------

uint64_t splitmix64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---- tree bookkeeping on the host -------------------------------------------------

uint64_t items_of(uint64_t N, int L, int lanes) {
  const uint64_t ch = (uint64_t)(8 / lanes) << (3 * L);  // executions per item
  const uint64_t it = (N + ch - 1) / ch;
  return it ? it : 1;
}

uint64_t groups_of(uint64_t N, int L) {
  uint64_t g = 0;
  for (int lvl = L; lvl < 19; ++lvl) g += N >> (3 * lvl + 3);
  return g;
}

// Tree-group slots any batch of `total_exec` executions can need at any chunk
// height: sum over strings of groups_of(N_i, 1) <= total_exec * (1/64 + 1/512
// + ...) < total_exec / 56.
static uint64_t groups_bound(uint64_t total_exec) { return total_exec / 56 + 1024; }

// Waits for the stream, then reads and clears a control block's status word
// (and, after a skipped out-of-range access in the checked build, the
// recorded kind and index).
int read_status(Ctl *ctl, cudaStream_t s) {
  HT_CUDA(cudaStreamSynchronize(s));
  unsigned int st = 0;
  HT_CUDA(cudaMemcpy(&st, &ctl->status, sizeof st, cudaMemcpyDeviceToHost));
  if (!st) return HT_OK;
  unsigned int kind = 0;
  unsigned long long index = 0;
  if (st & kStatusBounds) {
    HT_CUDA(cudaMemcpy(&kind, &ctl->bad_kind, sizeof kind, cudaMemcpyDeviceToHost));
    HT_CUDA(cudaMemcpy(&index, &ctl->bad_index, sizeof index, cudaMemcpyDeviceToHost));
    HT_CUDA(cudaMemset(&ctl->bad_kind, 0, sizeof kind));
    HT_CUDA(cudaMemset(&ctl->bad_index, 0, sizeof index));
  }
  HT_CUDA(cudaMemset(&ctl->status, 0, sizeof st));
  if (st & kStatusBounds) {
    static const char *const names[] = {"?", "input", "tree keys", "final-NH keys", "tail keys",
                                        "tree-group slot", "string slot", "digest row", "stack slot",
                                        "chunk buffer"};
    return set_error(HT_ERR_DEVICE, "checked build: an access outside its buffer was skipped (%s, index %llu)",
                     names[kind < 10 ? kind : 0], index);
  }
  if (st & kStatusTooLong)
    return set_error(HT_ERR_TOO_LONG, "a batch exceeded the reserved scratch (no digests written)");
  return set_error(HT_ERR_DEVICE, "a kernel gave up waiting for a shared-memory stage (status %u)", st);
}

static int bucket_of(uint64_t len) {
  if (len == UINT64_MAX) return 64;
  int b = 0;
  while (len > 1) {
    len >>= 1;
    ++b;
  }
  return b;
}

// ---- context ----------------------------------------------------------------------

static void free_scratch(ht_ctx *c) {
  cudaFree(c->grp_acc);
  cudaFree(c->grp_cnt);
  cudaFree(c->str_acc);
  cudaFree(c->str_done);
  cudaFree(c->plans);
  cudaFree(c->item0s);
  cudaFree(c->chunk0s);
  cudaFree(c->unitb0s);
  cudaFree(c->tile_items);
  cudaFree(c->tile_groups);
  cudaFree(c->tile_flags);
  cudaFree(c->item_str);
  c->tile_items = c->tile_groups = nullptr;
  c->tile_flags = nullptr;
  c->item_str = nullptr;
  c->cap_items = 0;
  c->chunk0s = nullptr;
  c->unitb0s = nullptr;
  c->grp_acc = nullptr;
  c->grp_cnt = nullptr;
  c->str_acc = nullptr;
  c->str_done = nullptr;
  c->plans = nullptr;
  c->item0s = nullptr;
  c->cap_groups = c->cap_strings = 0;
}

// Allocates zeroed scratch for `groups` tree groups and `strings` strings.
static int alloc_scratch(ht_ctx *c, uint64_t groups, uint64_t strings) {
  groups = std::max<uint64_t>(groups, 64);
  strings = std::max<uint64_t>(strings, 1);
  const size_t k = (size_t)c->ks->k;
  cudaError_t e = cudaSuccess;
  auto grab = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  };
  grab((void **)&c->grp_acc, groups * k * 8 * sizeof(unsigned long long));
  grab((void **)&c->grp_cnt, groups * sizeof(unsigned int));
  grab((void **)&c->str_acc, strings * k * sizeof(unsigned long long));
  grab((void **)&c->str_done, strings * sizeof(unsigned int));
  grab((void **)&c->plans, strings * sizeof(StrPlan));
  grab((void **)&c->item0s, (strings + 1) * sizeof(unsigned long long));
  grab((void **)&c->chunk0s, (strings + 1) * sizeof(unsigned long long));
  grab((void **)&c->unitb0s, (strings + 1) * sizeof(unsigned long long));
  const uint64_t tiles = (strings + 1023) / 1024 + 1;
  grab((void **)&c->tile_items, tiles * sizeof(unsigned long long));
  grab((void **)&c->tile_groups, tiles * sizeof(unsigned long long));
  grab((void **)&c->tile_flags, tiles * sizeof(unsigned int));
  // the item -> string map of warp-chunk batches with 64-execution (or
  // larger) items: a string of N executions has at most 1 + N/64 <=
  // 9 + 8 groups_of(N) items, so any batch that fits the group slots fits
  const uint64_t items = 8 * groups + 9 * strings;
  grab((void **)&c->item_str, items * sizeof(unsigned int));
  if (e != cudaSuccess) {
    free_scratch(c);
    return cuda_error(e, "scratch allocation");
  }
  c->cap_groups = groups;
  c->cap_strings = strings;
  c->cap_items = items;
  return HT_OK;
}

// Makes sure a single string of N executions fits the scratch (synchronous
// growth; rare).
static int ensure_groups(ht_ctx *c, uint64_t groups_needed, cudaStream_t s) {
  if (groups_needed <= c->cap_groups) return HT_OK;
  HT_CUDA(cudaStreamSynchronize(s));
  HT_CUDA(cudaDeviceSynchronize());
  const uint64_t strings = c->cap_strings;
  free_scratch(c);
  for (auto &g : c->graphs) g.valid = false;
  return alloc_scratch(c, groups_needed + groups_needed / 4, strings);
}

// Zeroes the tree-group slots, the string sums and counts and the control
// words (synchronous).
static int reset_scratch(ht_ctx *c, cudaStream_t s) {
  const size_t k = (size_t)c->ks->k;
  HT_CUDA(cudaMemsetAsync(c->grp_acc, 0, c->cap_groups * k * 8 * sizeof(unsigned long long), s));
  HT_CUDA(cudaMemsetAsync(c->grp_cnt, 0, c->cap_groups * sizeof(unsigned int), s));
  HT_CUDA(cudaMemsetAsync(c->str_acc, 0, c->cap_strings * k * sizeof(unsigned long long), s));
  HT_CUDA(cudaMemsetAsync(c->str_done, 0, c->cap_strings * sizeof(unsigned int), s));
  HT_CUDA(cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s));
  HT_CUDA(cudaStreamSynchronize(s));
  return HT_OK;
}

static Scratch scratch_view(const ht_ctx *c) {
  Scratch s;
  s.grp_acc = c->grp_acc;
  s.grp_cnt = c->grp_cnt;
  s.str_acc = c->str_acc;
  s.str_done = c->str_done;
  s.ctl = c->ctl;
  s.cap_groups = c->cap_groups;
  s.cap_strings = c->cap_strings;
  return s;
}

void fill_keys(const ht_ctx *c, KParams &P) {
  const KernelSet &ks = *c->ks;
  memset(&P, 0, sizeof P);
  for (int i = 0; i < ks.ew; ++i) P.E[i] = c->h_seeds[i];
  if (ks.tree) {
    // binary-tree ablation: level keys k_0 .. k_7 of every tree
    for (int t = 0; t < ks.k; ++t)
      for (int i = 0; i < 8; ++i) P.T0[t][i] = c->h_seeds[ks.off_T + t * kBinLevels + i];
  } else {
    for (int t = 0; t < ks.k; ++t)
      for (int i = 0; i < 7; ++i) P.T0[t][i] = c->h_seeds[ks.off_T + t * 19 * 7 + i];
  }
  P.seeds = c->d_seeds;
  P.scr = scratch_view(c);
  P.wait_cycles = c->wait_cycles;
}

// Dynamic shared memory of a stream-kernel block: per warp, `stages` slots of
// 8 executions plus one 8-byte mbarrier per slot, rounded to 128 bytes.
static size_t stream_smem(const KernelSet &ks, const ht_shape &s) {
  const size_t slot = 8 * (size_t)ks.exec_bytes;
  const size_t per_warp = ((size_t)s.stages * (slot + 8) + 127) & ~(size_t)127;
  return per_warp * (size_t)(s.threads_per_block / 32);
}

// Blocks per SM a kernel reaches (0 if it cannot run at all).
static int occupancy(const void *func, int tpb, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, tpb, smem) != cudaSuccess) n = 0;
  return n;
}

// The same, remembered by the context.
static int occupancy(ht_ctx *c, const void *func, int tpb, size_t smem) {
  for (const auto &o : c->occ_cache)
    if (o.func == func && o.tpb == tpb && o.smem == smem) return o.blocks;
  const int n = occupancy(func, tpb, smem);
  c->occ_cache.push_back({func, tpb, smem, n});
  return n;
}

// The warp-chunk kernel with 64-execution chunks measured fastest on GB300
// for long strings (the autotuner confirms or overrides per length bucket).
static ht_shape default_shape() {
  ht_shape s;
  s.kernel = 1;
  s.chunk_levels = 2;
  s.stages = 3;
  s.threads_per_block = 256;
  s.blocks_per_sm = 2;
  return s;
}

// Strings below 32 MiB (length buckets up to 24) take the block-chunk
// kernel where the kernel set has it: one execution per thread instead of
// eight in a row, and level 2 in shared memory.  Measured on GB300 (widths
// 24 and 40, back-to-back launches): 1 MiB 8.3-10.3 us (8-execution warp
// chunks 10.3-12.3, 64-execution warp chunks 16.4-17.9), 16 MiB 12.3-14.3
// (14.5-16.4, 21.2-22.5); from 32 MiB on 64-execution warp chunks are
// faster.
static ht_shape default_shape(const KernelSet &ks, int bucket) {
  ht_shape s = default_shape();
  if (bucket <= 24 && ks.block_single) s.kernel = 3;
  return s;
}

static bool shape_ok(const KernelSet &ks, const ht_shape &s) {
  if (s.threads_per_block < 32 || s.threads_per_block % 32 != 0 || s.blocks_per_sm < 1 ||
      s.blocks_per_sm > 32)
    return false;
  // 256-bit blocks and the binary-tree ablation: the warp-chunk kernel with
  // 64-execution items only
  if (ks.lanes != kLanes || ks.tree) return s.kernel == 1 && s.chunk_levels == 2 && s.threads_per_block <= 256;
  if (s.kernel == 0) return s.stages >= 2 && s.stages <= 8 && s.threads_per_block <= 256;
  if (s.kernel == 1)
    return s.chunk_levels >= 1 && s.chunk_levels <= 3 && s.threads_per_block <= 256;
  // block-chunk kernel: eight warps per block, single strings only
  if (s.kernel == 3) return ks.block_single != nullptr && s.threads_per_block == 256;
  return s.kernel == 2 && s.threads_per_block <= 256;
}

// Work units of a string for a shape: stream/range units (8 executions each,
// plus the tail unit) or warp-chunk items (8^L executions each, two
// 64-execution sub-chunks with 256-bit blocks; at least one).
static uint64_t units_for(const KernelSet &ks, const ht_shape &s, uint64_t N) {
  if (s.kernel == 3) return items_of(N, 2);  // block-chunk: 64-execution chunks
  return s.kernel != 1 ? ((N + 7) >> 3) + 1 : items_of(N, s.chunk_levels, ks.lanes);
}
static uint64_t unit_bytes(const KernelSet &ks, const ht_shape &s) {
  if (s.kernel == 3) return (uint64_t)ks.exec_bytes << 6;
  if (s.kernel != 1) return (uint64_t)ks.exec_bytes << 3;
  return ((uint64_t)ks.exec_bytes * (uint64_t)(kLanes / ks.lanes)) << (3 * s.chunk_levels);
}
static uint64_t groups_for(const KernelSet &ks, const ht_shape &s, uint64_t N) {
  if (ks.tree) return bin_groups(N);
  if (s.kernel == 3) return groups_of(N, 2);
  return groups_of(N, s.kernel != 1 ? 1 : s.chunk_levels);
}

// ---- single-string launch -------------------------------------------------------

// The kernel of a shape for a string.
static const void *single_func(const KernelSet &ks, const ht_shape &shape, const StrPlan &sp) {
  const bool al = (((uintptr_t)sp.ptr) & 15u) == 0;
  switch (shape.kernel) {
    case 0: return ks.stream_single;
    case 2: return al ? ks.range_single : ks.range_single_unaligned;
    case 3: return al ? ks.block_single : ks.block_single_unaligned;
    default: return al ? ks.single_aligned[shape.chunk_levels - 1] : ks.single_unaligned[shape.chunk_levels - 1];
  }
}

// Grid of one launch over `items` work items: blocks of *tpb threads (the
// block-chunk kernel: one item per block; the warp-chunk kernel: one item
// per warp, in whole rounds, a single round spread over every SM; stream
// and hybrid kernels: a few units per warp).
static uint64_t grid_for(const ht_ctx *c, int kernel, uint64_t items, int bps, int *tpb) {
  uint64_t wpb = (uint64_t)*tpb / 32;
  const uint64_t per_warp = kernel == 0 || kernel == 2 ? 4 : 1;
  const uint64_t want = kernel == 3 ? items : (items + per_warp * wpb - 1) / (per_warp * wpb);
  uint64_t grid = std::min<uint64_t>((uint64_t)c->num_sms * bps, want);
  if (kernel == 3) {
    // whole rounds of blocks, as below for warps
    const uint64_t bmax = (uint64_t)c->num_sms * bps;
    const uint64_t rounds = (items + bmax - 1) / bmax;
    grid = std::min(grid, (items + rounds - 1) / rounds);
  }
  if (kernel == 1) {
    // whole rounds: with R = ceil(items / max warps) rounds of cursor
    // grabs, ceil(items / R) warps finish together instead of a last round
    // that only a few warps work on
    const uint64_t wmax = (uint64_t)c->num_sms * bps * wpb;
    const uint64_t rounds = (items + wmax - 1) / wmax;
    const uint64_t warps = (items + rounds - 1) / rounds;
    grid = std::min(grid, (warps + wpb - 1) / wpb);
    if (rounds == 1 && grid < (uint64_t)c->num_sms) {
      // one round on fewer blocks than SMs: smaller blocks spread it over
      // every SM
      wpb = std::max<uint64_t>(1, warps / (uint64_t)c->num_sms);
      *tpb = (int)(32 * wpb);
      grid = (warps + wpb - 1) / wpb;
    }
  }
  return std::max<uint64_t>(grid, 1);
}

static int launch_kernel(const void *func, uint64_t grid, int tpb, size_t smem, KParams &P, bool pdl,
                         cudaStream_t s) {
  void *args[] = {&P};
  if (pdl) {
    // programmatic dependent launch: may start while the kernel before it in
    // the stream is still running (the kernel waits where that matters)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(tpb);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HT_CUDA(cudaLaunchKernelExC(&cfg, func, args));
  } else {
    HT_CUDA(cudaLaunchKernel(func, dim3((unsigned)grid), dim3(tpb), args, smem, s));
  }
  return HT_OK;
}

// Launches the kernel of a shape over units [u_begin, u_end) of the string
// described by sp (sp.n_items = all units of the string).  digest_dev
// receives k words when the string's last unit completes.
int launch_single(ht_ctx *c, const ht_shape &shape, const StrPlan &sp, uint64_t u_begin,
                  uint64_t u_end, uint64_t *digest_dev, cudaStream_t s) {
  const KernelSet &ks = *c->ks;
  const void *func = single_func(ks, shape, sp);
  const size_t smem = shape.kernel == 0 ? stream_smem(ks, shape) : 0;
  int tpb = shape.threads_per_block;
  const int occ = occupancy(c, func, tpb, smem);
  if (occ == 0) return set_error(HT_ERR_ARG, "launch shape does not fit the device");
  const int bps = std::min(shape.blocks_per_sm, occ);
  const uint64_t grid = grid_for(c, shape.kernel, u_end - u_begin, bps, &tpb);
  const bool overlap = (shape.kernel == 1 || shape.kernel == 3) && (c->flags & HT_FLAG_OVERLAP_LAUNCHES);
  KParams P;
  fill_keys(c, P);
  P.single = sp;
  P.item_begin = u_begin;
  P.item_end = u_end;
  P.digests = (unsigned long long *)digest_dev;
  P.count = 1;
  P.total_warps = (unsigned)(grid * (uint64_t)(tpb / 32));
  P.stages = (unsigned)shape.stages;
  int rc = launch_kernel(func, grid, tpb, smem, P, overlap, s);
  if (rc) return rc;
  c->launches.fetch_add(1);
  return HT_OK;
}

// Candidate launch shapes that fit the device, for single strings or for
// batches: the warp-chunk kernel (64-execution items only, for 256-bit
// blocks and for the binary-tree ablation) and, for single strings, the
// block-chunk kernel.
static std::vector<ht_shape> tune_candidates(ht_ctx *c, bool batch) {
  const KernelSet &ks = *c->ks;
  std::vector<ht_shape> cands;
  // (The stream and hybrid families are not candidates: on GB300 neither won
  // any length from 64 KiB to 1 GiB at widths 24 and 40, nor the
  // 50,000-string batch, timed on cold data; ht_set_shape still selects
  // them.)
  if (!batch && ks.block_single) {
    for (int bps : {1, 2, 3, 4, 6, 8}) {
      ht_shape h = default_shape();
      h.kernel = 3;
      h.threads_per_block = 256;
      h.blocks_per_sm = bps;
      if (occupancy(c, ks.block_single, 256, 0) < bps) continue;
      cands.push_back(h);
    }
  }
  for (int L : {1, 2, 3})
    for (int tpb : {128, 256})
      for (int bps : {1, 2, 3, 4, 6, 8}) {
        ht_shape h = default_shape();
        h.kernel = 1;
        h.chunk_levels = L;
        h.threads_per_block = tpb;
        h.blocks_per_sm = bps;
        const void *f = batch ? ks.batch[L - 1] : ks.single_aligned[L - 1];
        if (!f || occupancy(c, f, tpb, 0) < bps) continue;
        cands.push_back(h);
      }
  return cands;
}

}  // namespace ht

using namespace ht;

// ---- C ABI ---------------------------------------------------------------------------

extern "C" {

int ht_last_error(char *buf, size_t n) {
  if (buf && n) {
    strncpy(buf, g_err_msg, n - 1);
    buf[n - 1] = 0;
  }
  return g_err_code;
}

size_t ht_seed_words(int width) {
  const KernelSet *ks = kernel_set(width);
  return ks ? (size_t)ks->n_seed : 0;
}

int ht_seed_expand(uint64_t seed64, int width, uint64_t *out, size_t n) {
  const size_t need = ht_seed_words(width);
  if (!need) return set_error(HT_ERR_WIDTH, "unsupported width %d", width);
  if (!out || n != need)
    return set_error(HT_ERR_ARG, "seed buffer must hold %zu words (got %zu)", need, n);
  uint64_t st = seed64;
  for (size_t i = 0; i < n; ++i) out[i] = splitmix64_next(&st);
  return HT_OK;
}

int ht_ctx_create(int width, const uint64_t *seed_words, size_t n_words, ht_stream_t stream,
                  ht_ctx **out) {
  const KernelSet *ks = kernel_set(width);
  if (!ks) return set_error(HT_ERR_WIDTH, "unsupported width %d", width);
  if (!seed_words || !out || n_words != (size_t)ks->n_seed)
    return set_error(HT_ERR_ARG, "ht_ctx_create: need %d seed words (got %zu)", ks->n_seed,
                     n_words);
  *out = nullptr;
  ht_ctx *c = new ht_ctx();
  c->width = width;
  c->ks = ks;
  c->h_seeds.assign(seed_words, seed_words + n_words);
  for (int i = 0; i < 65; ++i) c->shapes[i] = i < 64 ? default_shape(*ks, i) : default_shape();
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_seeds, n_words * sizeof(uint64_t));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_seeds, seed_words, n_words * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_digest, 8 * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e == cudaSuccess && ks->stream_single)
    e = cudaFuncSetAttribute(ks->stream_single, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess && ks->stream_batch)
    e = cudaFuncSetAttribute(ks->stream_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  c->smem_optin = optin;
  if (e != cudaSuccess) {
    int rc = cuda_error(e, "ht_ctx_create");
    ht_ctx_destroy(c);
    return rc;
  }
  // default reserve: 16 GiB over at most 65536 strings
  int rc = alloc_scratch(c, groups_bound((16ull << 30) / (uint64_t)ks->exec_bytes), 65536);
  if (rc != HT_OK) {
    ht_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return HT_OK;
}

int ht_ctx_destroy(ht_ctx *c) {
  if (!c) return HT_OK;
  cudaDeviceSynchronize();
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  free_scratch(c);
  cudaFree(c->d_seeds);
  cudaFree(c->ctl);
  cudaFree(c->d_digest);
  for (int i = 0; i < kStageSlots; ++i) {
    cudaFree(c->stage[i]);
    if (c->ev_copy[i]) cudaEventDestroy(c->ev_copy[i]);
    if (c->ev_hash[i]) cudaEventDestroy(c->ev_hash[i]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->part_owned) cudaFree(c->part_buf);
  delete c;
  return HT_OK;
}

int ht_ctx_rekey(ht_ctx *c, const uint64_t *seed_words, size_t n_words, ht_stream_t stream) {
  if (!c || !seed_words || n_words != c->h_seeds.size())
    return set_error(HT_ERR_ARG, "ht_ctx_rekey: need %zu seed words", c ? c->h_seeds.size() : 0);
  // the previous upload may still be read by enqueued work: wait for it
  HT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  c->h_seeds.assign(seed_words, seed_words + n_words);
  HT_CUDA(cudaMemcpyAsync(c->d_seeds, c->h_seeds.data(), n_words * sizeof(uint64_t),
                          cudaMemcpyHostToDevice, (cudaStream_t)stream));
  HT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return HT_OK;
}

int ht_ctx_reserve(ht_ctx *c, uint64_t max_total_bytes, size_t max_strings) {
  if (!c || max_strings == 0) return set_error(HT_ERR_ARG, "ht_ctx_reserve: bad arguments");
  HT_CUDA(cudaDeviceSynchronize());
  free_scratch(c);
  for (auto &g : c->graphs) g.valid = false;
  return alloc_scratch(c, groups_bound(max_total_bytes / (uint64_t)c->ks->exec_bytes), max_strings);
}

int ht_ctx_status(ht_ctx *c, ht_stream_t stream) {
  if (!c) return set_error(HT_ERR_ARG, "ht_ctx_status: NULL context");
  const int rc = read_status(c->ctl, (cudaStream_t)stream);
  if (rc == HT_ERR_DEVICE) {
    // a kernel that gave up (a wait that ran out, an access the checked build
    // skipped) can leave tree groups, string sums and the cursor half
    // written: clear the scratch so that the next call starts clean
    char msg[256];
    ht_last_error(msg, sizeof msg);
    const int rr = reset_scratch(c, (cudaStream_t)stream);
    if (rr) return rr;
    return set_error(rc, "%s", msg);
  }
  return rc;
}

int ht_testing_set_wait_cycles(ht_ctx *c, uint64_t cycles) {
  if (!c || cycles > (1ull << 34)) return set_error(HT_ERR_ARG, "ht_testing_set_wait_cycles: bad arguments");
  c->wait_cycles = (long long)cycles;
  return HT_OK;
}

int ht_hash(ht_ctx *c, const void *data, uint64_t len, uint64_t *digest, ht_stream_t stream) {
  if (!c || !digest || (len && !data)) return set_error(HT_ERR_ARG, "ht_hash: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const ht_shape shape = c->shapes[bucket_of(len)];
  StrPlan sp;
  sp.ptr = (const uint8_t *)data;
  sp.len = len;
  sp.n_exec = len / (uint64_t)c->ks->exec_bytes;
  sp.item0 = 0;
  sp.grp0 = 0;
  const uint64_t n_units = units_for(*c->ks, shape, sp.n_exec);
  if (n_units > 0xffffffffull) return set_error(HT_ERR_TOO_LONG, "string too long for one launch");
  sp.n_items = (uint32_t)n_units;
  sp.pad = 0;
  int rc = ensure_groups(c, groups_for(*c->ks, shape, sp.n_exec), s);
  if (rc) return rc;
  return launch_single(c, shape, sp, 0, n_units, digest, s);
}

int ht_hash_host(ht_ctx *c, const void *data, uint64_t len, uint64_t *digest_host,
                 ht_stream_t stream) {
  if (!c || !digest_host || (len && !data)) return set_error(HT_ERR_ARG, "ht_hash_host: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const KernelSet &ks = *c->ks;
  const ht_shape shape = c->shapes[bucket_of(len)];
  const uint64_t B = (uint64_t)ks.exec_bytes;
  const uint64_t ub = unit_bytes(ks, shape);
  // pieces of whole units, about 64 MiB each (whole 64-execution chunks for
  // the unit-based kernels); a slot also holds the tail
  uint64_t units_per_piece = std::max<uint64_t>(1, (64ull << 20) / ub);
  if (shape.kernel == 0 || shape.kernel == 2) units_per_piece = std::max<uint64_t>(8, units_per_piece & ~7ull);
  const uint64_t slot_bytes = ((units_per_piece * ub + B + 255) / 256) * 256;
  if (!c->copy_stream) HT_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  if (c->stage_bytes < slot_bytes) {
    HT_CUDA(cudaDeviceSynchronize());
    for (int i = 0; i < kStageSlots; ++i) {
      cudaFree(c->stage[i]);
      c->stage[i] = nullptr;
    }
    for (int i = 0; i < kStageSlots; ++i) HT_CUDA(cudaMalloc((void **)&c->stage[i], slot_bytes));
    c->stage_bytes = slot_bytes;
  }
  for (int i = 0; i < kStageSlots; ++i) {
    if (!c->ev_copy[i]) HT_CUDA(cudaEventCreateWithFlags(&c->ev_copy[i], cudaEventDisableTiming));
    if (!c->ev_hash[i]) HT_CUDA(cudaEventCreateWithFlags(&c->ev_hash[i], cudaEventDisableTiming));
  }
  StrPlan sp;
  sp.len = len;
  sp.n_exec = len / B;
  sp.item0 = 0;
  sp.grp0 = 0;
  const uint64_t n_units = units_for(ks, shape, sp.n_exec);
  if (n_units > 0xffffffffull) return set_error(HT_ERR_TOO_LONG, "string too long for one launch");
  sp.n_items = (uint32_t)n_units;
  sp.pad = 0;
  int rc = ensure_groups(c, groups_for(*c->ks, shape, sp.n_exec), s);
  if (rc) return rc;
  // slots may still be read by an earlier call's kernels on another stream
  HT_CUDA(cudaStreamSynchronize(s));
  const uint8_t *host = (const uint8_t *)data;
  const uint64_t data_end = sp.n_exec * B;  // bytes read by EHC
  uint64_t piece = 0;
  for (uint64_t u0 = 0; u0 < n_units; u0 += units_per_piece, ++piece) {
    const uint64_t u1 = std::min(n_units, u0 + units_per_piece);
    // bytes of units [u0, u1); the last piece also carries the tail
    const uint64_t b0 = std::min(u0 * ub, data_end);
    const uint64_t b1 = (u1 == n_units) ? len : std::min(u1 * ub, data_end);
    const int slot = (int)(piece % kStageSlots);
    if (piece >= (uint64_t)kStageSlots) HT_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_hash[slot], 0));
    if (b1 > b0)
      HT_CUDA(cudaMemcpyAsync(c->stage[slot], host + b0, b1 - b0, cudaMemcpyHostToDevice, c->copy_stream));
    HT_CUDA(cudaEventRecord(c->ev_copy[slot], c->copy_stream));
    HT_CUDA(cudaStreamWaitEvent(s, c->ev_copy[slot], 0));
    // the kernel addresses the string from its start; shift the base so
    // that byte b0 lands at the slot
    sp.ptr = c->stage[slot] - b0;
    rc = launch_single(c, shape, sp, u0, u1, c->d_digest, s);
    if (rc) return rc;
    HT_CUDA(cudaEventRecord(c->ev_hash[slot], s));
  }
  HT_CUDA(cudaMemcpyAsync(digest_host, c->d_digest, (size_t)ks.k * 8, cudaMemcpyDeviceToHost, s));
  HT_CUDA(cudaStreamSynchronize(s));
  return HT_OK;
}

// The batch graph: planner nodes -> hash node(s).  The warp-chunk and
// stream kernels take the multi-block planner (tiles -> totals -> write, one
// thread per string) for batches of more than 1024 strings, and the
// one-block planner (one launch instead of three) for smaller ones; the
// hybrid kernel always takes the one-block planner, which also lays out its
// two-phase work list.  Each size class has a graph of its own, so that
// small and large batches alternating (a server) rebuild nothing.  Node
// parameters are replaced on every call; a graph is rebuilt when the batch
// shape changes.
struct BatchNodes {
  cudaKernelNodeParams plan, totals, write, items, hash, hash2;
  void *pargs[1], *hargs[1];
  bool multi;   // multi-block planner
  bool general; // a general (unaligned-capable) batch kernel follows the aligned-only one
  bool map;     // the planner writes the item -> string map (warp-chunk kernel, L >= 2)
};

// The general (unaligned-capable) batch kernel paired with the aligned-only
// one of a shape (none for the stream kernel, which handles both).
static const void *general_batch_kernel(const ht_ctx *c, const ht_shape &shape, bool map) {
  if (shape.kernel == 2) return c->ks->range_batch_unaligned;
  return map ? c->ks->batch_unaligned_map[shape.chunk_levels - 1] : c->ks->batch_unaligned[shape.chunk_levels - 1];
}

// Batches of at least this many strings find each work item's string in an
// item map that a fourth planner kernel writes (one load per item instead of
// a 32-way search over the prefix sums, 3 to 4 dependent loads at these
// sizes).  Measured on GB300: 2-3 % faster for 50,000 strings of up to
// 1 MiB and for 200,000 short strings; batches of a few thousand large
// strings (serving) are faster with the search (the search kernel keeps
// its code, the map costs a launch).
constexpr size_t kMapMinStrings = 16384;

// Whether a batch of `count` strings under `shape` uses the item map.
static bool use_map(const ht_ctx *c, const ht_shape &shape, size_t count) {
  return shape.kernel == 1 && shape.chunk_levels >= 2 && count >= kMapMinStrings &&
         c->ks->batch_map[shape.chunk_levels - 1] != nullptr;
}

// Batches of at most this many strings take the one-block planner (512-bit
// blocks and the paper's tree: its kernels lay out those plans only).
constexpr size_t kSmallBatch = 1024;

static bool small_batch(const ht_ctx *c, size_t count) {
  return count <= kSmallBatch && c->ks->lanes == kLanes && !c->ks->tree;
}

static void batch_nodes(ht_ctx *c, const ht_shape &shape, BatchNodes &n, bool small) {
  const KernelSet &ks = *c->ks;
  const int pl = shape.kernel == 1 ? shape.chunk_levels : 0;
  n.multi = shape.kernel != 2 && !small;
  n.general = shape.kernel != 0;
  n.map = use_map(c, shape, c->plan_args.count);
  c->plan_args.item_str = n.map ? c->item_str : nullptr;
  c->plan_args.cap_items = n.map ? c->cap_items : 0;
  c->batch_params.item_str = n.map ? c->item_str : nullptr;
  n.pargs[0] = &c->plan_args;
  const unsigned tiles = std::max(1u, (c->plan_args.count + 1023) / 1024);
  c->plan_args.n_tiles = tiles;
  n.plan = {};
  n.plan.blockDim = dim3(1024);
  n.plan.kernelParams = n.pargs;
  if (n.multi) {
    n.plan.func = (void *)ks.plan_tiles[pl];
    n.plan.gridDim = dim3(tiles);
    n.totals = n.plan;
    n.totals.func = (void *)ks.plan_totals;
    n.totals.gridDim = dim3(1);
    n.write = n.plan;
    n.write.func = (void *)ks.plan_write[pl];
    n.items = n.plan;
    n.items.func = (void *)ks.plan_items;
    n.items.gridDim = dim3((unsigned)(2 * c->num_sms));
    n.items.blockDim = dim3(256);
  } else {
    n.plan.func = (void *)ks.plan[pl];
    n.plan.gridDim = dim3(1);
  }
  n.hash = {};
  size_t smem = 0;
  const void *func;
  if (shape.kernel == 0) {
    func = ks.stream_batch;
    smem = stream_smem(ks, shape);
  } else if (shape.kernel == 2) {
    func = ks.range_batch;
  } else {
    func = n.map ? ks.batch_map[shape.chunk_levels - 1] : ks.batch[shape.chunk_levels - 1];
  }
  const int tpb = shape.threads_per_block;
  const int bps = std::max(1, std::min(shape.blocks_per_sm, occupancy(c, func, tpb, smem)));
  n.hash.func = (void *)func;
  n.hash.gridDim = dim3((unsigned)(c->num_sms * bps));
  n.hash.blockDim = dim3(tpb);
  n.hash.sharedMemBytes = (unsigned)smem;
  c->batch_params.total_warps = (unsigned)(c->num_sms * bps * (tpb / 32));
  c->batch_params.stages = (unsigned)shape.stages;
  c->plan_args.total_warps = c->batch_params.total_warps;
  n.hargs[0] = &c->batch_params;
  n.hash.kernelParams = n.hargs;
  n.hash2 = n.hash;
  if (n.general) n.hash2.func = (void *)general_batch_kernel(c, shape, n.map);
}

static int build_batch_graph(ht_ctx *c, const ht_shape &shape, bool small) {
  ht_ctx::BatchGraph &g = c->graphs[small ? 0 : 1];
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g = ht_ctx::BatchGraph();
  BatchNodes n;
  batch_nodes(c, shape, n, small);
  HT_CUDA(cudaGraphCreate(&g.graph, 0));
  HT_CUDA(cudaGraphAddKernelNode(&g.node_plan, g.graph, nullptr, 0, &n.plan));
  cudaGraphNode_t last = g.node_plan;
  if (n.multi) {
    HT_CUDA(cudaGraphAddKernelNode(&g.node_totals, g.graph, &last, 1, &n.totals));
    last = g.node_totals;
    HT_CUDA(cudaGraphAddKernelNode(&g.node_write, g.graph, &last, 1, &n.write));
    last = g.node_write;
    if (n.map) {
      HT_CUDA(cudaGraphAddKernelNode(&g.node_items, g.graph, &last, 1, &n.items));
      last = g.node_items;
    }
  }
  HT_CUDA(cudaGraphAddKernelNode(&g.node_hash, g.graph, &last, 1, &n.hash));
  if (n.general) {
    // the general variant; the one the planner's flag does not select
    // returns at once
    HT_CUDA(cudaGraphAddKernelNode(&g.node_hash2, g.graph, &g.node_hash, 1, &n.hash2));
  }
  HT_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
  g.shape = shape;
  g.map = n.map;
  g.valid = true;
  return HT_OK;
}

int ht_hash_batch(ht_ctx *c, const void *const *ptrs, const uint64_t *lens, size_t count,
                  uint64_t *digests, ht_stream_t stream) {
  if (!c || (count && (!ptrs || !lens || !digests)))
    return set_error(HT_ERR_ARG, "ht_hash_batch: bad arguments");
  if (count == 0) return HT_OK;
  if (count > c->cap_strings)
    return set_error(HT_ERR_TOO_LONG, "batch of %zu strings above the reserve (%llu)", count,
                     (unsigned long long)c->cap_strings);
  cudaStream_t s = (cudaStream_t)stream;
  const ht_shape shape = c->shapes[64];
  PlanArgs &A = c->plan_args;
  A.ptrs = ptrs;
  A.lens = lens;
  A.count = (unsigned)count;
  A.plans = c->plans;
  A.item0s = c->item0s;
  A.chunk0s = c->chunk0s;
  A.unitb0s = c->unitb0s;
  A.ctl = c->ctl;
  A.cap_groups = c->cap_groups;
  A.tile_items = c->tile_items;
  A.tile_groups = c->tile_groups;
  A.tile_flags = c->tile_flags;
  KParams &P = c->batch_params;
  fill_keys(c, P);
  P.plans = c->plans;
  P.item0s = c->item0s;
  P.chunk0s = c->chunk0s;
  P.unitb0s = c->unitb0s;
  P.digests = (unsigned long long *)digests;
  P.count = (unsigned)count;
  const bool small = small_batch(c, count);
  ht_ctx::BatchGraph &g = c->graphs[small ? 0 : 1];
  if (!g.valid || memcmp(&g.shape, &shape, sizeof shape) != 0 || g.map != use_map(c, shape, count)) {
    int rc = build_batch_graph(c, shape, small);
    if (rc) return rc;
  } else {
    BatchNodes n;
    batch_nodes(c, shape, n, small);
    HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_plan, &n.plan));
    if (g.node_totals) HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_totals, &n.totals));
    if (g.node_write) HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_write, &n.write));
    if (g.node_items) HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_items, &n.items));
    HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_hash, &n.hash));
    if (g.node_hash2) HT_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.node_hash2, &n.hash2));
  }
  HT_CUDA(cudaGraphLaunch(g.exec, s));
  c->launches.fetch_add(2 + (g.node_totals ? 2 : 0) + (g.node_items ? 1 : 0) + (g.node_hash2 ? 1 : 0));
  return HT_OK;
}

int ht_hash_batch_naive(ht_ctx *c, const void *const *ptrs_host, const uint64_t *lens_host,
                        size_t count, uint64_t *digests, ht_stream_t stream) {
  if (!c || (count && (!ptrs_host || !lens_host || !digests)))
    return set_error(HT_ERR_ARG, "ht_hash_batch_naive: bad arguments");
  const int k = c->ks->k;
  for (size_t i = 0; i < count; ++i) {
    int rc = ht_hash(c, ptrs_host[i], lens_host[i], digests + i * (size_t)k, stream);
    if (rc) return rc;
  }
  return HT_OK;
}

int ht_ctx_set_flags(ht_ctx *c, unsigned flags) {
  if (!c || (flags & ~(unsigned)HT_FLAG_OVERLAP_LAUNCHES))
    return set_error(HT_ERR_ARG, "ht_ctx_set_flags: unknown flags %u", flags);
  c->flags = flags;
  return HT_OK;
}

int ht_get_shape(ht_ctx *c, uint64_t len, ht_shape *out) {
  if (!c || !out) return set_error(HT_ERR_ARG, "ht_get_shape: bad arguments");
  *out = c->shapes[bucket_of(len)];
  return HT_OK;
}

int ht_set_shape(ht_ctx *c, uint64_t len, const ht_shape *shape) {
  if (!c || !shape || !shape_ok(*c->ks, *shape) || (len == UINT64_MAX && shape->kernel == 3))
    return set_error(HT_ERR_ARG, "ht_set_shape: bad shape");
  c->shapes[bucket_of(len)] = *shape;
  return HT_OK;
}

uint64_t ht_ctx_launches(ht_ctx *c) { return c ? c->launches.load() : 0; }

unsigned ht_build_flags(void) { return kChecked ? HT_BUILD_CHECKED : 0u; }

int ht_wait_probe(ht_ctx *c, uint64_t cycles, ht_stream_t stream) {
  if (!c || cycles == 0 || cycles > (1ull << 34)) return set_error(HT_ERR_ARG, "ht_wait_probe: bad arguments");
  if (!c->ks->wait_probe) return set_error(HT_ERR_WIDTH, "ht_wait_probe: the binary-tree ablation has no staged kernel");
  Ctl *ctl = c->ctl;
  long long budget = (long long)cycles;
  void *args[] = {&ctl, &budget};
  HT_CUDA(cudaLaunchKernel(c->ks->wait_probe, dim3(1), dim3(32), args, 0, (cudaStream_t)stream));
  return HT_OK;
}

int ht_check_probe(ht_ctx *c, uint64_t index, uint64_t limit, ht_stream_t stream) {
  if (!c) return set_error(HT_ERR_ARG, "ht_check_probe: NULL context");
  check_probe_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(c->ctl, index, limit);
  HT_CUDA(cudaGetLastError());
  return HT_OK;
}

int ht_autotune(ht_ctx *c, uint64_t len, ht_stream_t stream, ht_shape *best) {
  if (!c || len == UINT64_MAX) return set_error(HT_ERR_ARG, "ht_autotune: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<ht_shape> cands = tune_candidates(c, false);
  // strings shorter than the L2 cache would be timed from L2: successive
  // launches take successive copies in a buffer of at least 384 MiB, so
  // that every launch reads its bytes from HBM, as a fresh request does
  const uint64_t stride = (std::max<uint64_t>(len, 16) + 255) & ~255ull;
  const uint64_t copies = std::max<uint64_t>(1, (384ull << 20) / stride);
  const uint64_t span = stride * copies;
  uint8_t *buf = nullptr;
  HT_CUDA(cudaMalloc((void **)&buf, span));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = HT_OK;
  cudaError_t ce = cudaMemsetAsync(buf, 0x5A, span, s);
  if (ce != cudaSuccess) rc = cuda_error(ce, "cudaMemsetAsync");
  const int bk = bucket_of(len);
  const ht_shape saved = c->shapes[bk];
  ht_shape winner = saved;
  float best_ms = 1e30f;
  uint64_t turn = 0;
  for (size_t i = 0; i < cands.size() && rc == HT_OK; ++i) {
    c->shapes[bk] = cands[i];
    rc = ht_hash(c, buf + (turn++ % copies) * stride, len, c->d_digest, stream);  // warm-up
    float times[3] = {0, 0, 0};
    for (int r = 0; r < 3 && rc == HT_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = ht_hash(c, buf + (turn++ % copies) * stride, len, c->d_digest, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&times[r], e0, e1);
    }
    if (rc) break;
    std::sort(times, times + 3);
    if (times[1] < best_ms) {
      best_ms = times[1];
      winner = cands[i];
    }
  }
  c->shapes[bk] = (rc == HT_OK) ? winner : saved;
  cudaStreamSynchronize(s);
  if (rc == HT_OK) {
    int st = ht_ctx_status(c, stream);
    if (st) rc = st;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc == HT_OK && best) *best = winner;
  return rc;
}

int ht_autotune_batch(ht_ctx *c, const void *const *ptrs, const uint64_t *lens, size_t count,
                      uint64_t *digests, ht_stream_t stream, ht_shape *best) {
  if (!c || count == 0 || !ptrs || !lens || !digests)
    return set_error(HT_ERR_ARG, "ht_autotune_batch: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<ht_shape> cands = tune_candidates(c, true);
  cudaEvent_t e0, e1;
  HT_CUDA(cudaEventCreate(&e0));
  HT_CUDA(cudaEventCreate(&e1));
  const ht_shape saved = c->shapes[64];
  ht_shape winner = saved;
  float best_ms = 1e30f;
  int rc = HT_OK;
  bool any = false;
  for (size_t i = 0; i < cands.size() && rc == HT_OK; ++i) {
    c->shapes[64] = cands[i];
    rc = ht_hash_batch(c, ptrs, lens, count, digests, stream);  // warm-up (builds the graph)
    if (rc) break;
    const int st = read_status(c->ctl, s);
    if (st == HT_ERR_TOO_LONG) continue;  // this chunk height needs more group slots
    if (st) {
      rc = st;
      break;
    }
    float times[3] = {0, 0, 0};
    for (int r = 0; r < 3 && rc == HT_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = ht_hash_batch(c, ptrs, lens, count, digests, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&times[r], e0, e1);
    }
    if (rc) break;
    std::sort(times, times + 3);
    any = true;
    if (times[1] < best_ms) {
      best_ms = times[1];
      winner = cands[i];
    }
  }
  if (rc == HT_OK && !any) rc = set_error(HT_ERR_TOO_LONG, "ht_autotune_batch: the batch fits no shape's scratch");
  c->shapes[64] = (rc == HT_OK) ? winner : saved;
  // the digests of the winning shape (every shape gives the same digests)
  if (rc == HT_OK) rc = ht_hash_batch(c, ptrs, lens, count, digests, stream);
  if (rc == HT_OK) rc = read_status(c->ctl, s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HT_OK && best) *best = winner;
  return rc;
}

}  // extern "C"
