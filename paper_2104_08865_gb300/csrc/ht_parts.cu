// ht_parts.cu -- host side of hashing one string in parts (see ht_parts.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "halftime.h"
#include "ht_internal.h"
#include "ht_runtime.h"
#include "ht_spec.cuh"

namespace {

constexpr int kPartLevels = 2;  // parts use the warp-chunk kernel, 64-execution chunks

// dst[i] += src[i] over a part state.
__global__ void part_merge_kernel(unsigned long long *dst, const unsigned long long *src, size_t words) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

// Words of a part state for N executions: 8 pending-root sums, one word for
// the unit count, the 32-bit arrival counters packed two per word, then the
// node accumulators.
struct PartLayout {
  uint64_t groups, cnt_words, words;
};

PartLayout part_layout(const ht::KernelSet &ks, uint64_t N) {
  PartLayout L;
  L.groups = ht::groups_of(N, kPartLevels);
  L.cnt_words = (L.groups + 1) / 2;
  L.words = 9 + L.cnt_words + L.groups * (uint64_t)ks.k * 8;
  return L;
}

void part_params(const ht_ctx *c, ht::KParams &P, uint64_t total_len) {
  const ht::KernelSet &ks = *c->ks;
  memset(&P, 0, sizeof P);
  for (int i = 0; i < ks.ew; ++i) P.E[i] = c->h_seeds[i];
  for (int t = 0; t < ks.k; ++t)
    for (int i = 0; i < 7; ++i) P.T0[t][i] = c->h_seeds[ks.off_T + t * 19 * 7 + i];
  P.seeds = c->d_seeds;
  const PartLayout L = part_layout(ks, total_len / (uint64_t)ks.exec_bytes);
  unsigned long long *b = c->part_buf;
  P.scr.str_acc = b;
  P.scr.str_done = reinterpret_cast<unsigned int *>(b + 8);
  P.scr.grp_cnt = reinterpret_cast<unsigned int *>(b + 9);
  P.scr.grp_acc = b + 9 + L.cnt_words;
  P.scr.ctl = c->ctl;
  P.scr.cap_groups = L.groups;
  P.scr.cap_strings = 1;
  ht::StrPlan &sp = P.single;
  sp.len = total_len;
  sp.n_exec = total_len / (uint64_t)ks.exec_bytes;
  sp.item0 = 0;
  sp.grp0 = 0;
  sp.n_items = 0xffffffffu;  // never reached: parts never run the finaliser
  P.count = 1;
}

}  // namespace

using namespace ht;

extern "C" {

uint64_t ht_part_granule(ht_ctx *c) {
  return c && c->ks->lanes == kLanes && !c->ks->tree ? (uint64_t)c->ks->exec_bytes << (3 * kPartLevels) : 0;
}

size_t ht_part_state_words(ht_ctx *c, uint64_t total_len) {
  return c && c->ks->lanes == kLanes && !c->ks->tree ? (size_t)part_layout(*c->ks, total_len / (uint64_t)c->ks->exec_bytes).words : 0;
}

int ht_part_begin(ht_ctx *c, uint64_t total_len, void *state_dev, size_t words, ht_stream_t stream) {
  if (!c) return set_error(HT_ERR_ARG, "ht_part_begin: NULL context");
  if (c->ks->lanes != kLanes || c->ks->tree)
    return set_error(HT_ERR_WIDTH, "ht_part_begin: parts take 512-bit blocks and the default tree");
  const PartLayout L = part_layout(*c->ks, total_len / (uint64_t)c->ks->exec_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  if (state_dev) {
    // the caller's buffer (for example a tensor it will all-reduce)
    if (words < L.words)
      return set_error(HT_ERR_ARG, "ht_part_begin: state buffer of %zu words, need %llu", words,
                       (unsigned long long)L.words);
    if (c->part_owned) cudaFree(c->part_buf);
    c->part_buf = static_cast<unsigned long long *>(state_dev);
    c->part_owned = false;
    c->part_cap_words = words;
  } else if (!c->part_owned || c->part_cap_words < L.words) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "ht_part_begin");
    if (c->part_owned) cudaFree(c->part_buf);
    c->part_buf = nullptr;
    c->part_cap_words = 0;
    e = cudaMalloc((void **)&c->part_buf, L.words * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_error(e, "part state allocation");
    c->part_owned = true;
    c->part_cap_words = L.words;
  }
  cudaError_t e = cudaMemsetAsync(c->part_buf, 0, L.words * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_error(e, "ht_part_begin");
  c->part_len = total_len;
  c->part_open = true;
  return HT_OK;
}

int ht_hash_part(ht_ctx *c, const void *part_dev, uint64_t part_offset, uint64_t part_len,
                 ht_stream_t stream) {
  if (!c || !c->part_open) return set_error(HT_ERR_ARG, "ht_hash_part: call ht_part_begin first");
  const uint64_t total = c->part_len;
  const uint64_t gran = ht_part_granule(c);
  if (part_offset > total || part_len > total - part_offset || (part_len && !part_dev))
    return set_error(HT_ERR_ARG, "ht_hash_part: part outside the string");
  const bool last = part_offset + part_len == total;
  if (part_offset % gran || (!last && part_len % gran))
    return set_error(HT_ERR_ARG, "ht_hash_part: parts must start and end on multiples of %llu bytes",
                     (unsigned long long)gran);
  KParams P;
  part_params(c, P, total);
  const uint64_t N = P.single.n_exec;
  const uint64_t n_items = items_of(N, kPartLevels);
  const uint64_t i0 = part_offset / gran;
  const uint64_t i1 = last ? n_items : (part_offset + part_len) / gran;
  P.single.ptr = static_cast<const uint8_t *>(part_dev) - part_offset;
  cudaStream_t s = (cudaStream_t)stream;
  if (i1 > i0) {
    const bool aligned = (((uintptr_t)P.single.ptr) & 15u) == 0;
    const void *func = aligned ? c->ks->single_aligned[kPartLevels - 1] : c->ks->single_unaligned[kPartLevels - 1];
    const int tpb = 256;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, func, tpb, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy");
    bps = std::max(bps, 1);
    const uint64_t wpb = tpb / 32;
    uint64_t grid = std::min<uint64_t>((uint64_t)c->num_sms * bps, (i1 - i0 + wpb - 1) / wpb);
    grid = std::max<uint64_t>(grid, 1);
    P.item_begin = i0;
    P.item_end = i1;
    P.total_warps = (unsigned)(grid * wpb);
    void *args[] = {&P};
    e = cudaLaunchKernel(func, dim3((unsigned)grid), dim3(tpb), args, 0, s);
    if (e != cudaSuccess) return cuda_error(e, "ht_hash_part launch");
    c->launches.fetch_add(1);
  }
  if (last) {
    void *args[] = {&P};
    cudaError_t e = cudaLaunchKernel(c->ks->part_tail, dim3(1), dim3(32), args, 0, s);
    if (e != cudaSuccess) return cuda_error(e, "ht_hash_part tail launch");
    c->launches.fetch_add(1);
  }
  return HT_OK;
}

int ht_part_state(ht_ctx *c, void **state_dev, size_t *words) {
  if (!c || !state_dev || !words || !c->part_open)
    return set_error(HT_ERR_ARG, "ht_part_state: no open part state");
  *state_dev = c->part_buf;
  *words = part_layout(*c->ks, c->part_len / (uint64_t)c->ks->exec_bytes).words;
  return HT_OK;
}

int ht_part_merge(ht_ctx *c, const void *state_dev, size_t words, ht_stream_t stream) {
  if (!c || !c->part_open || !state_dev)
    return set_error(HT_ERR_ARG, "ht_part_merge: bad arguments");
  const size_t mine = part_layout(*c->ks, c->part_len / (uint64_t)c->ks->exec_bytes).words;
  if (words != mine) return set_error(HT_ERR_ARG, "ht_part_merge: state of %zu words, expected %zu", words, mine);
  const unsigned grid = (unsigned)std::min<size_t>((words + 255) / 256, 4096);
  part_merge_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(
      c->part_buf, static_cast<const unsigned long long *>(state_dev), words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "ht_part_merge launch");
  c->launches.fetch_add(1);
  return HT_OK;
}

int ht_finish_parts(ht_ctx *c, uint64_t *digest_dev, ht_stream_t stream) {
  if (!c || !c->part_open || !digest_dev) return set_error(HT_ERR_ARG, "ht_finish_parts: bad arguments");
  KParams P;
  part_params(c, P, c->part_len);
  P.digests = reinterpret_cast<unsigned long long *>(digest_dev);
  void *args[] = {&P};
  cudaError_t e = cudaLaunchKernel(c->ks->part_finish, dim3(1), dim3(32), args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "ht_finish_parts launch");
  c->launches.fetch_add(1);
  c->part_open = false;
  return HT_OK;
}

}  // extern "C"
