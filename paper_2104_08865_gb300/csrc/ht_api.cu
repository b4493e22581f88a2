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
#include "ht_internal.h"
#include "ht_runtime.h"

namespace ht {

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
    default: return nullptr;
  }
}

// ---- seeds: splitmix64 (Steele, Lea, Flood 2014) ------------------------------

static uint64_t splitmix64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---- tree bookkeeping on the host -------------------------------------------------

uint64_t items_of(uint64_t N, int L) {
  const uint64_t it = (N + (1ull << (3 * L)) - 1) >> (3 * L);
  return it ? it : 1;
}

uint64_t groups_of(uint64_t N, int L) {
  uint64_t g = 0;
  for (int lvl = L; lvl < 19; ++lvl) g += N >> (3 * lvl + 3);
  return g;
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
  if (e != cudaSuccess) {
    free_scratch(c);
    return cuda_error(e, "scratch allocation");
  }
  c->cap_groups = groups;
  c->cap_strings = strings;
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
  c->graph_valid = false;
  return alloc_scratch(c, groups_needed + groups_needed / 4, strings);
}

static Scratch scratch_view(const ht_ctx *c) {
  Scratch s;
  s.grp_acc = c->grp_acc;
  s.grp_cnt = c->grp_cnt;
  s.str_acc = c->str_acc;
  s.str_done = c->str_done;
  s.ctl = c->ctl;
  s.cap_groups = c->cap_groups;
  return s;
}

static void fill_keys(const ht_ctx *c, KParams &P) {
  const KernelSet &ks = *c->ks;
  memset(&P, 0, sizeof P);
  for (int i = 0; i < ks.ew; ++i) P.E[i] = c->h_seeds[i];
  for (int t = 0; t < ks.k; ++t)
    for (int i = 0; i < 7; ++i) P.T0[t][i] = c->h_seeds[ks.off_T + t * 19 * 7 + i];
  P.seeds = c->d_seeds;
  P.scr = scratch_view(c);
}

// Blocks per SM a kernel reaches with tpb threads (at least 1).
static int occupancy(const void *func, int tpb) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, tpb, 0) != cudaSuccess) n = 1;
  return std::max(n, 1);
}

static ht_shape default_shape() {
  ht_shape s;
  s.chunk_levels = 2;
  s.threads_per_block = 256;
  s.blocks_per_sm = 32;  // clamped to occupancy at launch
  return s;
}

static bool shape_ok(const ht_shape &s) {
  return (s.chunk_levels == 2 || s.chunk_levels == 3) && s.threads_per_block >= 32 &&
         s.threads_per_block <= 256 && s.threads_per_block % 32 == 0 && s.blocks_per_sm >= 1 &&
         s.blocks_per_sm <= 32;
}

// ---- single-string launch -------------------------------------------------------

// Launches the single-string kernel over items [item_begin, item_end) of the
// string described by sp.  digest_dev receives k words when the string's last
// item completes.
int launch_single(ht_ctx *c, const ht_shape &shape, const StrPlan &sp,
                  uint64_t item_begin, uint64_t item_end, uint64_t *digest_dev,
                  cudaStream_t s) {
  const KernelSet &ks = *c->ks;
  const int L = shape.chunk_levels;
  const bool aligned = (((uintptr_t)sp.ptr) & 15u) == 0;
  const void *func = aligned ? ks.single_aligned[L - 2] : ks.single_unaligned[L - 2];
  const int tpb = shape.threads_per_block;
  const int bps = std::min(shape.blocks_per_sm, occupancy(func, tpb));
  const uint64_t warps_needed = item_end - item_begin;
  const uint64_t wpb = (uint64_t)tpb / 32;
  uint64_t grid = std::min<uint64_t>((uint64_t)c->num_sms * bps, (warps_needed + wpb - 1) / wpb);
  grid = std::max<uint64_t>(grid, 1);
  KParams P;
  fill_keys(c, P);
  P.single = sp;
  P.item_begin = item_begin;
  P.item_end = item_end;
  P.digests = (unsigned long long *)digest_dev;
  P.count = 1;
  P.total_warps = (unsigned)(grid * wpb);
  void *args[] = {&P};
  HT_CUDA(cudaLaunchKernel(func, dim3((unsigned)grid), dim3(tpb), args, 0, s));
  c->launches.fetch_add(1);
  return HT_OK;
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
  for (int i = 0; i < 65; ++i) c->shapes[i] = default_shape();
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
  if (e != cudaSuccess) {
    int rc = cuda_error(e, "ht_ctx_create");
    ht_ctx_destroy(c);
    return rc;
  }
  // default reserve: 64 GiB over at most 65536 strings
  const uint64_t total_exec = (64ull << 30) / (uint64_t)ks->exec_bytes;
  int rc = alloc_scratch(c, total_exec / 448 + 1024, 65536);
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
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
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
  const uint64_t total_exec = max_total_bytes / (uint64_t)c->ks->exec_bytes;
  free_scratch(c);
  c->graph_valid = false;
  return alloc_scratch(c, total_exec / 448 + 1024, max_strings);
}

int ht_ctx_status(ht_ctx *c, ht_stream_t stream) {
  if (!c) return set_error(HT_ERR_ARG, "ht_ctx_status: NULL context");
  HT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned int st = 0;
  HT_CUDA(cudaMemcpy(&st, &c->ctl->status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) {
    unsigned int zero = 0;
    HT_CUDA(cudaMemcpy(&c->ctl->status, &zero, sizeof zero, cudaMemcpyHostToDevice));
    return set_error(HT_ERR_TOO_LONG, "a batch exceeded the reserved scratch (no digests written)");
  }
  return HT_OK;
}

int ht_hash(ht_ctx *c, const void *data, uint64_t len, uint64_t *digest, ht_stream_t stream) {
  if (!c || !digest || (len && !data)) return set_error(HT_ERR_ARG, "ht_hash: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const ht_shape shape = c->shapes[bucket_of(len)];
  const int L = shape.chunk_levels;
  StrPlan sp;
  sp.ptr = (const uint8_t *)data;
  sp.len = len;
  sp.n_exec = len / (uint64_t)c->ks->exec_bytes;
  sp.item0 = 0;
  sp.grp0 = 0;
  const uint64_t n_items = items_of(sp.n_exec, L);
  if (n_items > 0xffffffffull) return set_error(HT_ERR_TOO_LONG, "string too long for one launch");
  sp.n_items = (uint32_t)n_items;
  sp.pad = 0;
  int rc = ensure_groups(c, groups_of(sp.n_exec, L), s);
  if (rc) return rc;
  return launch_single(c, shape, sp, 0, n_items, digest, s);
}

int ht_hash_host(ht_ctx *c, const void *data, uint64_t len, uint64_t *digest_host,
                 ht_stream_t stream) {
  if (!c || !digest_host || (len && !data)) return set_error(HT_ERR_ARG, "ht_hash_host: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const KernelSet &ks = *c->ks;
  const ht_shape shape = c->shapes[bucket_of(len)];
  const int L = shape.chunk_levels;
  const uint64_t B = (uint64_t)ks.exec_bytes;
  const uint64_t chunk_bytes = B << (3 * L);
  // pieces of whole chunks, about 64 MiB each; a slot also holds the tail
  const uint64_t items_per_piece = std::max<uint64_t>(1, (64ull << 20) / chunk_bytes);
  const uint64_t slot_bytes = ((items_per_piece * chunk_bytes + B + 255) / 256) * 256;
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
  const uint64_t n_items = items_of(sp.n_exec, L);
  if (n_items > 0xffffffffull) return set_error(HT_ERR_TOO_LONG, "string too long for one launch");
  sp.n_items = (uint32_t)n_items;
  sp.pad = 0;
  int rc = ensure_groups(c, groups_of(sp.n_exec, L), s);
  if (rc) return rc;
  // slots may still be read by an earlier call's kernels on another stream
  HT_CUDA(cudaStreamSynchronize(s));
  const uint8_t *host = (const uint8_t *)data;
  uint64_t piece = 0;
  for (uint64_t it0 = 0; it0 < n_items; it0 += items_per_piece, ++piece) {
    const uint64_t it1 = std::min(n_items, it0 + items_per_piece);
    const uint64_t b0 = it0 * chunk_bytes;
    const uint64_t b1 = (it1 == n_items) ? len : it1 * chunk_bytes;
    const int slot = (int)(piece % kStageSlots);
    if (piece >= (uint64_t)kStageSlots) HT_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_hash[slot], 0));
    if (b1 > b0)
      HT_CUDA(cudaMemcpyAsync(c->stage[slot], host + b0, b1 - b0, cudaMemcpyHostToDevice, c->copy_stream));
    HT_CUDA(cudaEventRecord(c->ev_copy[slot], c->copy_stream));
    HT_CUDA(cudaStreamWaitEvent(s, c->ev_copy[slot], 0));
    // the kernel addresses the string from its start; shift the base so
    // that byte b0 lands at the slot
    sp.ptr = c->stage[slot] - b0;
    rc = launch_single(c, shape, sp, it0, it1, c->d_digest, s);
    if (rc) return rc;
    HT_CUDA(cudaEventRecord(c->ev_hash[slot], s));
  }
  HT_CUDA(cudaMemcpyAsync(digest_host, c->d_digest, (size_t)ks.k * 8, cudaMemcpyDeviceToHost, s));
  HT_CUDA(cudaStreamSynchronize(s));
  return HT_OK;
}

static int build_batch_graph(ht_ctx *c, const ht_shape &shape) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  const KernelSet &ks = *c->ks;
  const int L = shape.chunk_levels;
  HT_CUDA(cudaGraphCreate(&c->graph, 0));
  cudaKernelNodeParams np = {};
  np.func = (void *)ks.plan[L - 2];
  np.gridDim = dim3(1);
  np.blockDim = dim3(1024);
  void *pargs[] = {&c->plan_args};
  np.kernelParams = pargs;
  HT_CUDA(cudaGraphAddKernelNode(&c->node_plan, c->graph, nullptr, 0, &np));
  cudaKernelNodeParams nh = {};
  const void *func = ks.batch[L - 2];
  const int tpb = shape.threads_per_block;
  const int bps = std::min(shape.blocks_per_sm, occupancy(func, tpb));
  nh.func = (void *)func;
  nh.gridDim = dim3((unsigned)(c->num_sms * bps));
  nh.blockDim = dim3(tpb);
  c->batch_params.total_warps = (unsigned)(c->num_sms * bps * (tpb / 32));
  void *hargs[] = {&c->batch_params};
  nh.kernelParams = hargs;
  HT_CUDA(cudaGraphAddKernelNode(&c->node_hash, c->graph, &c->node_plan, 1, &nh));
  HT_CUDA(cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
  c->node_hash_params = nh;
  c->graph_shape = shape;
  c->graph_valid = true;
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
  const KernelSet &ks = *c->ks;
  PlanArgs &A = c->plan_args;
  A.ptrs = ptrs;
  A.lens = lens;
  A.count = (unsigned)count;
  A.plans = c->plans;
  A.item0s = c->item0s;
  A.ctl = c->ctl;
  A.cap_groups = c->cap_groups;
  KParams &P = c->batch_params;
  fill_keys(c, P);
  P.plans = c->plans;
  P.item0s = c->item0s;
  P.digests = (unsigned long long *)digests;
  P.count = (unsigned)count;
  const int L = shape.chunk_levels;
  const void *func = ks.batch[L - 2];
  const int bps = std::min(shape.blocks_per_sm, occupancy(func, shape.threads_per_block));
  P.total_warps = (unsigned)(c->num_sms * bps * (shape.threads_per_block / 32));
  if (!c->graph_valid || memcmp(&c->graph_shape, &shape, sizeof shape) != 0) {
    int rc = build_batch_graph(c, shape);
    if (rc) return rc;
  } else {
    cudaKernelNodeParams np = {};
    np.func = (void *)ks.plan[L - 2];
    np.gridDim = dim3(1);
    np.blockDim = dim3(1024);
    void *pargs[] = {&c->plan_args};
    np.kernelParams = pargs;
    HT_CUDA(cudaGraphExecKernelNodeSetParams(c->graph_exec, c->node_plan, &np));
    cudaKernelNodeParams nh = c->node_hash_params;
    void *hargs[] = {&c->batch_params};
    nh.kernelParams = hargs;
    HT_CUDA(cudaGraphExecKernelNodeSetParams(c->graph_exec, c->node_hash, &nh));
  }
  HT_CUDA(cudaGraphLaunch(c->graph_exec, s));
  c->launches.fetch_add(2);
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

int ht_get_shape(ht_ctx *c, uint64_t len, ht_shape *out) {
  if (!c || !out) return set_error(HT_ERR_ARG, "ht_get_shape: bad arguments");
  *out = c->shapes[bucket_of(len)];
  return HT_OK;
}

int ht_set_shape(ht_ctx *c, uint64_t len, const ht_shape *shape) {
  if (!c || !shape || !shape_ok(*shape)) return set_error(HT_ERR_ARG, "ht_set_shape: bad shape");
  c->shapes[bucket_of(len)] = *shape;
  return HT_OK;
}

uint64_t ht_ctx_launches(ht_ctx *c) { return c ? c->launches.load() : 0; }

int ht_autotune(ht_ctx *c, uint64_t len, ht_stream_t stream, ht_shape *best) {
  if (!c || len == UINT64_MAX) return set_error(HT_ERR_ARG, "ht_autotune: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *buf = nullptr;
  HT_CUDA(cudaMalloc((void **)&buf, std::max<uint64_t>(len, 16)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = HT_OK;
  cudaError_t ce = cudaMemsetAsync(buf, 0x5A, std::max<uint64_t>(len, 16), s);
  if (ce != cudaSuccess) rc = cuda_error(ce, "cudaMemsetAsync");
  const ht_shape saved = c->shapes[bucket_of(len)];
  ht_shape winner = saved;
  float best_ms = 1e30f;
  const int Ls[2] = {2, 3};
  const int tpbs[2] = {128, 256};
  const int bpss[6] = {1, 2, 3, 4, 6, 8};
  for (int li = 0; li < 2 && rc == HT_OK; ++li)
    for (int ti = 0; ti < 2 && rc == HT_OK; ++ti)
      for (int bi = 0; bi < 6 && rc == HT_OK; ++bi) {
        ht_shape cand;
        cand.chunk_levels = Ls[li];
        cand.threads_per_block = tpbs[ti];
        cand.blocks_per_sm = bpss[bi];
        const void *func = c->ks->single_aligned[cand.chunk_levels - 2];
        if (cand.blocks_per_sm > occupancy(func, cand.threads_per_block)) continue;
        c->shapes[bucket_of(len)] = cand;
        rc = ht_hash(c, buf, len, c->d_digest, stream);  // warm-up
        if (rc) break;
        float times[3];
        for (int r = 0; r < 3 && rc == HT_OK; ++r) {
          cudaEventRecord(e0, s);
          rc = ht_hash(c, buf, len, c->d_digest, stream);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&times[r], e0, e1);
        }
        if (rc) break;
        std::sort(times, times + 3);
        if (times[1] < best_ms) {
          best_ms = times[1];
          winner = cand;
        }
      }
  c->shapes[bucket_of(len)] = (rc == HT_OK) ? winner : saved;
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc == HT_OK && best) *best = winner;
  return rc;
}

}  // extern "C"
