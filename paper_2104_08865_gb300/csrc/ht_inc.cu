// ht_inc.cu -- incremental hashing: a string given in pieces of any length,
// one after another, whose total length is known only at the end.
//
// The handle holds the string's eager tree counter between calls (Section
// 5.2: the pending nodes of every level, kept on a stack) and a buffer for
// bytes that do not yet fill a 64-execution chunk.  Updates run the
// block-chunk kernel (below 32 MiB) or the warp-chunk kernel in its
// incremental mode over whole chunks, straight from the caller's memory; only the bytes after an update's last whole chunk
// are copied (by the update kernel itself, into the handle's other buffer),
// and the next update reads its first chunk from the buffer and from its
// own first bytes, so that an update is one kernel that may overlap the one
// before it.  The final call hashes the stack's pending nodes, the buffered
// executions and the tail.  The digest equals the one-shot digest of the
// concatenated pieces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "halftime.h"
#include "ht_internal.h"
#include "ht_runtime.h"
#include "ht_spec.cuh"

using namespace ht;

namespace {

constexpr int kChunkExecs = 64;             // executions per chunk (a level-2 node)
constexpr uint64_t kMaxChunks = 1u << 16;   // chunks per update launch
constexpr uint64_t kStageChunks = 1024;     // chunks per staging slot of host updates
constexpr int kStageSlots2 = 2;
constexpr uint64_t kStateMagic = 0x31636e4948544831ull;  // "1HTHInc1"
constexpr int kTpb = 256;

// Group slots an update of chunks [C, C + M) can complete: at level l >= 2,
// the groups between the ones holding node C >> 3(l-2) and node
// (C + M) >> 3(l-2).
uint64_t groups_for_update(uint64_t C, uint64_t M) {
  uint64_t g = 0;
  const uint64_t N0 = C * kChunkExecs, N1 = (C + M) * kChunkExecs;
  for (int lvl = 2; lvl < kLevels - 1; ++lvl) g += ((N1 >> (3 * lvl)) >> 3) - ((N0 >> (3 * lvl)) >> 3);
  return g;
}

uint64_t seed_fingerprint(const ht_ctx *c) {
  uint64_t h = 0xcbf29ce484222325ull;  // FNV-1a over the seed words' bytes
  for (uint64_t w : c->h_seeds)
    for (int i = 0; i < 8; ++i) {
      h ^= (w >> (8 * i)) & 0xff;
      h *= 0x100000001b3ull;
    }
  return h;
}

}  // namespace

struct ht_inc {
  ht_ctx *ctx = nullptr;
  int k = 0;
  uint64_t granule = 0;  // bytes of one chunk
  uint64_t cap_groups = 0;
  // device state
  unsigned long long *grp_acc = nullptr;
  unsigned int *grp_cnt = nullptr;
  unsigned long long *str_acc = nullptr;
  unsigned int *str_done = nullptr;
  Ctl *ctl = nullptr;
  unsigned long long *stack[2] = {nullptr, nullptr};  // the state and the next update's output
  int cur = 0;            // stack[cur] holds the state
  // bytes short of a whole chunk wait in buf[bcur]; an update's kernel
  // copies its own remainder into the other buffer (so that it never writes
  // the buffer it reads its first chunk from)
  uint8_t *buf[2] = {nullptr, nullptr};
  int bcur = 0;
  // host mirror of the counter
  uint64_t chunks = 0;  // whole chunks hashed
  uint64_t fill = 0;    // bytes waiting in buf (< granule)
  bool open = false;
  // host updates: staging slots filled on a copy stream
  cudaStream_t copy_stream = nullptr;
  uint8_t *stage[kStageSlots2] = {nullptr, nullptr};
  cudaEvent_t ev_copy[kStageSlots2] = {nullptr, nullptr};
  cudaEvent_t ev_hash[kStageSlots2] = {nullptr, nullptr};
  uint64_t piece = 0;
};

namespace {

size_t stack_words(const ht_inc *h) { return (size_t)kLevels * kFan * h->k * kLanes; }

void inc_params(const ht_inc *h, KParams &P) {
  fill_keys(h->ctx, P);
  P.scr.grp_acc = h->grp_acc;
  P.scr.grp_cnt = h->grp_cnt;
  P.scr.str_acc = h->str_acc;
  P.scr.str_done = h->str_done;
  P.scr.ctl = h->ctl;
  P.scr.cap_groups = h->cap_groups;
  P.scr.cap_strings = 1;
  P.stack = h->stack[h->cur];
  P.stack_in = h->stack[h->cur];
  P.count = 1;
}

// Updates of fewer bytes than this run the block-chunk kernel (a block of
// eight warps per chunk, one execution per thread; its block for the first
// chunk reads it with 256 threads), longer ones the warp-chunk kernel (with
// eight warps on a first chunk read from two places).  Measured on GB300
// (width 24, pieces back to back with overlapping launches, us per update):
// 16 MiB + 3 bytes 11.3 (block) / 11.2 (warp), 32 MiB + 3 15.6 / 15.6,
// 64 MiB + 3 24.3 / 17.7, 780 whole chunks 22.7 / 15.7, 128 MiB + 3
// 29.0 / 28.8.
constexpr uint64_t kBlockwiseBytes = 32ull << 20;

// Hashes chunks [h->chunks, h->chunks + M): the first from the chunk buffer
// if first_from_buf, the others (or all) contiguous at ptr (device).  One
// launch; it reads the stack of the state and writes the other one, and
// copies rem_len bytes from rem_src into the other chunk buffer (which then
// becomes the current one).  fill > 0: the buffer holds only the first
// fill bytes of the first chunk, and the launch reads its other G - fill
// bytes where they are, before ptr.  pdl: launched to overlap the kernel
// before it.
int run_chunks(ht_inc *h, bool first_from_buf, const uint8_t *ptr, uint64_t M, cudaStream_t s,
               const uint8_t *rem_src = nullptr, uint64_t rem_len = 0, bool pdl = false,
               uint64_t fill = 0) {
  ht_ctx *c = h->ctx;
  const KernelSet &ks = *c->ks;
  const uint64_t C = h->chunks;
  // (the last slot is the first chunk's level-1 group of warp-chunk updates
  // that read that chunk from two places)
  if (groups_for_update(C, M) > h->cap_groups - 1)
    return set_error(HT_ERR_ARG, "incremental update needs more group slots than reserved");
  KParams P;
  inc_params(h, P);
  P.stack_in = h->stack[h->cur];
  P.stack = h->stack[h->cur ^ 1];
  StrPlan &sp = P.single;
  // the kernel addresses the string from its start
  sp.ptr = ptr - (C + (first_from_buf ? 1 : 0)) * h->granule;
  if (first_from_buf) P.inc_first = h->buf[h->bcur];
  P.inc_fill = first_from_buf ? fill : 0;
  // (the update's first G - fill bytes end where the chunks at ptr begin)
  P.inc_stage_src = (unsigned long long)(uintptr_t)(ptr - (h->granule - fill));
  P.inc_rem_src = rem_src;
  P.inc_rem_dst = h->buf[h->bcur ^ 1];
  P.inc_rem_len = rem_len;
  sp.n_exec = (C + M) * kChunkExecs;
  sp.len = sp.n_exec * (uint64_t)ks.exec_bytes;
  sp.chunk0 = C;
  sp.n_items = 0xffffffffu;
  void *args[] = {&P};
  // (a partial buffered chunk takes the update's first bytes at any
  // alignment: the general kernel)
  const bool aligned = (((uintptr_t)sp.ptr) & 15u) == 0 && !P.inc_fill;
  const bool blockwise = M * h->granule < kBlockwiseBytes;
  const void *func = blockwise ? (aligned ? ks.inc_block_aligned : ks.inc_block_unaligned)
                               : (aligned ? ks.inc_aligned : ks.inc_unaligned);
  const int bps = 2;  // (both kernels fit two blocks of 256 threads per SM)
  uint64_t wpb = kTpb / 32, grid;
  if (blockwise) {
    // one chunk per block, whole rounds of blocks, and one more block that
    // seeds the frontier
    const uint64_t bmax = (uint64_t)c->num_sms * bps;
    const uint64_t rounds = (M + bmax - 1) / bmax;
    grid = (M + rounds - 1) / rounds + 1;
  } else {
    // whole rounds of cursor grabs (see the one-shot launch), one round
    // spread over every SM, and one more warp that seeds the frontier; a
    // first chunk read from two places goes to eight warps of its own
    const uint64_t Mc = M - (P.inc_fill ? 1 : 0);  // chunks from the cursor
    const uint64_t wmax = (uint64_t)c->num_sms * bps * wpb;
    const uint64_t rounds = std::max<uint64_t>(1, (Mc + wmax - 1) / wmax);
    const uint64_t warps = (Mc + rounds - 1) / rounds + (P.inc_fill ? 9 : 1);
    grid = std::max<uint64_t>(1, (warps + wpb - 1) / wpb);
    if (rounds == 1 && grid < (uint64_t)c->num_sms) {
      wpb = std::max<uint64_t>(1, warps / (uint64_t)c->num_sms);
      grid = (warps + wpb - 1) / wpb;
    }
  }
  grid = std::max<uint64_t>(grid, 1);
  P.item_begin = C + (!blockwise && P.inc_fill ? 1 : 0);
  P.item_end = C + M;
  P.inc_chunk0_slot = h->cap_groups - 1;
  P.total_warps = (unsigned)(grid * wpb);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)(32 * wpb));
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelExC(&cfg, func, args);
  if (e != cudaSuccess) return cuda_error(e, "incremental update launch");
  c->launches.fetch_add(1);
  h->chunks = C + M;
  h->cur ^= 1;
  if (rem_len) h->bcur ^= 1;
  return HT_OK;
}

void free_inc(ht_inc *h) {
  cudaFree(h->grp_acc);
  cudaFree(h->grp_cnt);
  cudaFree(h->str_acc);
  cudaFree(h->str_done);
  cudaFree(h->ctl);
  cudaFree(h->stack[0]);
  cudaFree(h->stack[1]);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  for (int i = 0; i < kStageSlots2; ++i) {
    cudaFree(h->stage[i]);
    if (h->ev_copy[i]) cudaEventDestroy(h->ev_copy[i]);
    if (h->ev_hash[i]) cudaEventDestroy(h->ev_hash[i]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
}

#define INC_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_error(e_, #call); \
  } while (0)

}  // namespace

extern "C" {

int ht_inc_create(ht_ctx *c, ht_inc **out) {
  if (!c || !out) return set_error(HT_ERR_ARG, "ht_inc_create: NULL argument");
  *out = nullptr;
  if (c->ks->lanes != kLanes || c->ks->tree)
    return set_error(HT_ERR_WIDTH, "ht_inc_create: incremental hashing takes 512-bit blocks");
  ht_inc *h = new ht_inc;
  h->ctx = c;
  h->k = c->ks->k;
  h->granule = (uint64_t)kChunkExecs * (uint64_t)c->ks->exec_bytes;
  h->cap_groups = kMaxChunks / 7 + 2 * kLevels;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(p, n);
  };
  alloc((void **)&h->grp_acc, h->cap_groups * h->k * kLanes * sizeof(unsigned long long));
  alloc((void **)&h->grp_cnt, h->cap_groups * sizeof(unsigned int));
  alloc((void **)&h->str_acc, 8 * sizeof(unsigned long long));
  alloc((void **)&h->str_done, 256);
  alloc((void **)&h->ctl, sizeof(Ctl));
  alloc((void **)&h->stack[0], stack_words(h) * sizeof(unsigned long long));
  alloc((void **)&h->stack[1], stack_words(h) * sizeof(unsigned long long));
  alloc((void **)&h->buf[0], h->granule);
  alloc((void **)&h->buf[1], h->granule);
  if (e != cudaSuccess) {
    free_inc(h);
    delete h;
    return cuda_error(e, "ht_inc_create allocation");
  }
  const int rc = ht_inc_init(h, nullptr);
  if (rc != HT_OK) {
    free_inc(h);
    delete h;
    return rc;
  }
  e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    free_inc(h);
    delete h;
    return cuda_error(e, "ht_inc_create");
  }
  *out = h;
  return HT_OK;
}

int ht_inc_destroy(ht_inc *h) {
  if (!h) return HT_OK;
  cudaDeviceSynchronize();
  free_inc(h);
  delete h;
  return HT_OK;
}

int ht_inc_init(ht_inc *h, ht_stream_t stream) {
  if (!h) return set_error(HT_ERR_ARG, "ht_inc_init: NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  INC_CUDA(cudaMemsetAsync(h->grp_acc, 0, h->cap_groups * h->k * kLanes * sizeof(unsigned long long), s));
  INC_CUDA(cudaMemsetAsync(h->grp_cnt, 0, h->cap_groups * sizeof(unsigned int), s));
  INC_CUDA(cudaMemsetAsync(h->str_acc, 0, 8 * sizeof(unsigned long long), s));
  INC_CUDA(cudaMemsetAsync(h->str_done, 0, 256, s));
  INC_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
  h->chunks = 0;
  h->fill = 0;
  h->bcur = 0;
  h->open = true;
  return HT_OK;
}

uint64_t ht_inc_length(const ht_inc *h) { return h ? h->chunks * h->granule + h->fill : 0; }

int ht_inc_status(ht_inc *h, ht_stream_t stream) {
  if (!h) return set_error(HT_ERR_ARG, "ht_inc_status: NULL handle");
  return read_status(h->ctl, (cudaStream_t)stream);
}

uint64_t ht_inc_granule(const ht_inc *h) { return h ? h->granule : 0; }

int ht_inc_update(ht_inc *h, const void *data_dev, uint64_t len, ht_stream_t stream) {
  if (!h || !h->open) return set_error(HT_ERR_ARG, "ht_inc_update: call ht_inc_init first");
  if (len && !data_dev) return set_error(HT_ERR_ARG, "ht_inc_update: NULL data");
  if (len > ~0ull - ht_inc_length(h)) return set_error(HT_ERR_TOO_LONG, "ht_inc_update: string longer than 2^64 - 1 bytes");
  cudaStream_t s = (cudaStream_t)stream;
  const uint8_t *p = static_cast<const uint8_t *>(data_dev);
  const uint64_t G = h->granule;
  uint64_t m = len;
  if (!m) return HT_OK;
  if (h->fill + m < G) {
    // no chunk completes: the bytes join the buffer
    INC_CUDA(cudaMemcpyAsync(h->buf[h->bcur] + h->fill, p, m, cudaMemcpyDeviceToDevice, s));
    h->fill += m;
    return HT_OK;
  }
  // kernels only (each update's remainder copied by the update itself), so
  // that with HT_FLAG_OVERLAP_LAUNCHES each may overlap the one before it
  const bool pdl = (h->ctx->flags & HT_FLAG_OVERLAP_LAUNCHES) != 0;
  // the first launch reads the partial chunk from the buffer and from the
  // update's first bytes
  const bool buffered0 = h->fill != 0;
  bool buffered = buffered0;
  const uint64_t fill = h->fill;
  if (buffered0) {
    p += G - fill;
    m -= G - fill;
  }
  uint64_t M = m / G;
  const uint64_t rem = m - M * G;
  while (buffered || M) {
    const uint64_t piece = std::min(M, kMaxChunks - (buffered ? 1 : 0));
    const bool last = piece == M;
    const int rc = run_chunks(h, buffered, p, piece + (buffered ? 1 : 0), s, last ? p + piece * G : nullptr,
                              last ? rem : 0, pdl, buffered ? fill : 0);
    if (rc) return rc;
    buffered = false;
    p += piece * G;
    M -= piece;
  }
  h->fill = rem;
  return HT_OK;
}

int ht_inc_update_host(ht_inc *h, const void *data_host, uint64_t len, ht_stream_t stream) {
  if (!h || !h->open) return set_error(HT_ERR_ARG, "ht_inc_update_host: call ht_inc_init first");
  if (len && !data_host) return set_error(HT_ERR_ARG, "ht_inc_update_host: NULL data");
  if (len > ~0ull - ht_inc_length(h))
    return set_error(HT_ERR_TOO_LONG, "ht_inc_update_host: string longer than 2^64 - 1 bytes");
  cudaStream_t s = (cudaStream_t)stream;
  const uint8_t *p = static_cast<const uint8_t *>(data_host);
  uint64_t m = len;
  bool buffered = false;  // the chunk buffer holds a whole chunk for the first launch
  if (h->fill) {
    const uint64_t r = std::min(m, h->granule - h->fill);
    if (r) INC_CUDA(cudaMemcpyAsync(h->buf[h->bcur] + h->fill, p, r, cudaMemcpyHostToDevice, s));
    h->fill += r;
    p += r;
    m -= r;
    if (h->fill < h->granule) {
      INC_CUDA(cudaStreamSynchronize(s));
      return HT_OK;
    }
    buffered = true;
  }
  uint64_t M = m / h->granule;
  if (M) {
    const uint64_t slot_bytes = kStageChunks * h->granule;
    if (!h->copy_stream) INC_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < kStageSlots2; ++i) {
      if (!h->stage[i]) INC_CUDA(cudaMalloc((void **)&h->stage[i], slot_bytes));
      if (!h->ev_copy[i]) INC_CUDA(cudaEventCreateWithFlags(&h->ev_copy[i], cudaEventDisableTiming));
      if (!h->ev_hash[i]) INC_CUDA(cudaEventCreateWithFlags(&h->ev_hash[i], cudaEventDisableTiming));
    }
    // pieces alternate between two slots: the copy of one overlaps the
    // hashing of the other
    while (M) {
      const uint64_t piece = std::min(M, kStageChunks);
      const int slot = (int)(h->piece++ % kStageSlots2);
      INC_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_hash[slot], 0));
      INC_CUDA(cudaMemcpyAsync(h->stage[slot], p, piece * h->granule, cudaMemcpyHostToDevice, h->copy_stream));
      INC_CUDA(cudaEventRecord(h->ev_copy[slot], h->copy_stream));
      INC_CUDA(cudaStreamWaitEvent(s, h->ev_copy[slot], 0));
      const int rc = run_chunks(h, buffered, h->stage[slot], piece + (buffered ? 1 : 0), s);
      if (rc) return rc;
      INC_CUDA(cudaEventRecord(h->ev_hash[slot], s));
      if (buffered) h->fill = 0;
      buffered = false;
      p += piece * h->granule;
      m -= piece * h->granule;
      M -= piece;
    }
  }
  if (buffered) {
    const int rc = run_chunks(h, true, h->buf[h->bcur], 1, s);
    if (rc) return rc;
    h->fill = 0;
  }
  if (m) {
    INC_CUDA(cudaMemcpyAsync(h->buf[h->bcur], p, m, cudaMemcpyHostToDevice, s));
    h->fill = m;
  }
  // the caller may reuse its buffer once this returns (copies from pinned
  // memory are asynchronous)
  INC_CUDA(cudaStreamSynchronize(s));
  return HT_OK;
}

int ht_inc_final(ht_inc *h, uint64_t *digest_dev, ht_stream_t stream) {
  if (!h || !h->open) return set_error(HT_ERR_ARG, "ht_inc_final: call ht_inc_init first");
  if (!digest_dev) return set_error(HT_ERR_ARG, "ht_inc_final: NULL digest");
  ht_ctx *c = h->ctx;
  const KernelSet &ks = *c->ks;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t C = h->chunks;
  KParams P;
  inc_params(h, P);
  StrPlan &sp = P.single;
  sp.ptr = h->buf[h->bcur] - C * h->granule;
  sp.len = C * h->granule + h->fill;
  sp.n_exec = C * kChunkExecs + h->fill / (uint64_t)ks.exec_bytes;
  sp.chunk0 = C;
  sp.n_items = 1;  // reached by the remainder launch below (items [C, C + 1)): it ends the string
  P.digests = reinterpret_cast<unsigned long long *>(digest_dev);
  void *args[] = {&P};
  if (C) {
    INC_CUDA(cudaLaunchKernel(ks.inc_stack, dim3(1), dim3(32), args, 0, s));
    c->launches.fetch_add(1);
  }
  // the buffered executions (fewer than one chunk: pending nodes of levels 0
  // and 1) and the tail, by the one-shot kernel's last chunk of the string
  P.item_begin = C;
  P.item_end = C + 1;
  P.total_warps = 1;
  INC_CUDA(cudaLaunchKernel(ks.single_aligned[1], dim3(1), dim3(32), args, 0, s));
  c->launches.fetch_add(1);
  h->open = false;
  return HT_OK;
}

size_t ht_inc_state_bytes(const ht_inc *h) {
  return h ? 4 * sizeof(uint64_t) + stack_words(h) * sizeof(uint64_t) + h->granule : 0;
}

int ht_inc_export(const ht_inc *h, void *state_host, size_t n, ht_stream_t stream) {
  if (!h || !h->open || !state_host) return set_error(HT_ERR_ARG, "ht_inc_export: no open string");
  if (n < ht_inc_state_bytes(h)) return set_error(HT_ERR_ARG, "ht_inc_export: buffer of %zu bytes, need %zu", n, ht_inc_state_bytes(h));
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t *hd = static_cast<uint64_t *>(state_host);
  hd[0] = kStateMagic ^ (uint64_t)h->ctx->width;
  hd[1] = seed_fingerprint(h->ctx);
  hd[2] = h->chunks;
  hd[3] = h->fill;
  uint8_t *b = static_cast<uint8_t *>(state_host) + 4 * sizeof(uint64_t);
  INC_CUDA(cudaMemcpyAsync(b, h->stack[h->cur], stack_words(h) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  if (h->fill)
    INC_CUDA(cudaMemcpyAsync(b + stack_words(h) * sizeof(uint64_t), h->buf[h->bcur], h->fill, cudaMemcpyDeviceToHost, s));
  INC_CUDA(cudaStreamSynchronize(s));
  return HT_OK;
}

int ht_inc_import(ht_inc *h, const void *state_host, size_t n, ht_stream_t stream) {
  if (!h || !state_host) return set_error(HT_ERR_ARG, "ht_inc_import: NULL argument");
  if (n < ht_inc_state_bytes(h)) return set_error(HT_ERR_ARG, "ht_inc_import: state of %zu bytes, need %zu", n, ht_inc_state_bytes(h));
  const uint64_t *hd = static_cast<const uint64_t *>(state_host);
  if (hd[0] != (kStateMagic ^ (uint64_t)h->ctx->width))
    return set_error(HT_ERR_ARG, "ht_inc_import: not a state of a width-%d string", h->ctx->width);
  if (hd[1] != seed_fingerprint(h->ctx))
    return set_error(HT_ERR_ARG, "ht_inc_import: the state was made with other seed words");
  if (hd[3] >= h->granule || hd[2] > (~0ull - hd[3]) / h->granule)
    return set_error(HT_ERR_ARG, "ht_inc_import: corrupt state");
  int rc = ht_inc_init(h, stream);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const uint8_t *b = static_cast<const uint8_t *>(state_host) + 4 * sizeof(uint64_t);
  INC_CUDA(cudaMemcpyAsync(h->stack[h->cur], b, stack_words(h) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  if (hd[3])
    INC_CUDA(cudaMemcpyAsync(h->buf[h->bcur], b + stack_words(h) * sizeof(uint64_t), hd[3], cudaMemcpyHostToDevice, s));
  INC_CUDA(cudaStreamSynchronize(s));
  h->chunks = hd[2];
  h->fill = hd[3];
  return HT_OK;
}

}  // extern "C"
