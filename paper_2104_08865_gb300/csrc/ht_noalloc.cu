// ht_noalloc.cu -- hashing one string without allocating any memory.
//
// Some callers cannot allocate device memory: code running inside another
// framework's allocator hooks (a cudaMalloc there would re-enter the
// allocator), processes whose device memory is already reserved by another
// framework's memory pool (an extra cudaMalloc fails or breaks that pool's
// accounting), and latency-critical paths that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  They cannot create an
// ht_ctx, whose constructor allocates.  ht_hash_noalloc serves them: the tree
// scratch (control words, completion counters, node accumulators) and the
// device copy of the seed words live in one file-scope __device__ array of
// fixed size that the library reserves at load time, and the caller passes
// only its inputs and outputs.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "halftime.h"
#include "ht_internal.h"
#include "ht_runtime.h"
#include "ht_spec.cuh"

namespace {

// Scratch of ht_hash_noalloc: 8 MiB, held by every GPU that loads the library
// until the process exits.
constexpr size_t kNoAllocBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Layout of the array (byte offsets, 256-byte aligned regions).
constexpr size_t kOffCtl = 0;
constexpr size_t kOffSeeds = 256;
constexpr size_t kSeedBytes = 57344;  // >= 6897 seed words (width 40)
static_assert(kSeedBytes >= ht::Dims<40>::n_seed * sizeof(uint64_t) &&
                  kSeedBytes >= ht::Dims<32>::n_seed * sizeof(uint64_t),
              "the seed region holds the largest seed layout");
constexpr size_t kOffStrAcc = kOffSeeds + kSeedBytes;
constexpr size_t kOffStrDone = kOffStrAcc + 256;
constexpr size_t kOffGroups = kOffStrDone + 256;
constexpr int kChunkLevels = 2;  // the warp-chunk kernel with 64-execution chunks

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (host code only holds a stand-in for the symbol, not its address).
// The same first call loads every kernel this entry point may launch, for
// every width: with lazy module loading a kernel's module is otherwise
// loaded, with driver-side allocations, at its first launch.
int scratch_on_current_device(unsigned char **addr, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ht::cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return ht::set_error(HT_ERR_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return ht::cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ht::cuda_error(e, "cudaDeviceGetAttribute");
    for (int w : {16, 24, 32, 40}) {
      const ht::KernelSet *ks = ht::kernel_set(w);
      for (const void *f : {ks->single_aligned[kChunkLevels - 1], ks->single_unaligned[kChunkLevels - 1]}) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return ht::cuda_error(e, "cudaFuncGetAttributes(no-alloc kernels)");
      }
    }
    g_addr[dev] = static_cast<unsigned char *>(p);
    g_sms[dev] = n;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return HT_OK;
}

// Tree groups the array holds for a width: a counter and a k x 8-word node
// accumulator each, after the fixed regions (256 bytes kept for rounding the
// counter region up).
uint64_t noalloc_max_groups(const ht::KernelSet &ks) {
  const size_t per_group = sizeof(unsigned int) + (size_t)ks.k * 8 * sizeof(unsigned long long);
  return (kNoAllocBytes - kOffGroups - 256) / per_group;
}

}  // namespace

extern "C" int ht_hash_noalloc(int width_bytes, const uint64_t *seed_words_host, size_t n_words,
                               const void *data_dev, uint64_t len, uint64_t *digest_dev,
                               ht_stream_t stream) {
  const ht::KernelSet *ks = ht::kernel_set(width_bytes);
  if (!ks || ks->lanes != ht::kLanes || ks->tree) return ht::set_error(HT_ERR_WIDTH, "unsupported width %d", width_bytes);
  if (!seed_words_host || n_words != (size_t)ks->n_seed || !digest_dev || (len && !data_dev) ||
      n_words * sizeof(uint64_t) > kSeedBytes)
    return ht::set_error(HT_ERR_ARG, "ht_hash_noalloc: bad arguments (need %d seed words)", ks->n_seed);
  const uint64_t N = len / (uint64_t)ks->exec_bytes;
  const uint64_t groups = ht::groups_of(N, kChunkLevels);
  const uint64_t max_groups = noalloc_max_groups(*ks);
  if (groups > max_groups)
    return ht::set_error(HT_ERR_TOO_LONG,
                         "ht_hash_noalloc: %llu bytes need %llu tree groups, the fixed scratch holds %llu",
                         (unsigned long long)len, (unsigned long long)groups,
                         (unsigned long long)max_groups);
  unsigned char *base = nullptr;
  int sms = 1;
  int rc = scratch_on_current_device(&base, &sms);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t k = (size_t)ks->k;
  unsigned int *grp_cnt = reinterpret_cast<unsigned int *>(base + kOffGroups);
  const size_t cnt_bytes = ((max_groups * sizeof(unsigned int)) + 255) & ~(size_t)255;
  unsigned long long *grp_acc = reinterpret_cast<unsigned long long *>(base + kOffGroups + cnt_bytes);
  // the seed words go next to the scratch; everything the kernel counts or
  // accumulates in must start at zero
  cudaError_t e = cudaMemcpyAsync(base + kOffSeeds, seed_words_host, n_words * sizeof(uint64_t),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffCtl, 0, sizeof(ht::Ctl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffStrAcc, 0, 512, s);
  if (e == cudaSuccess && groups) e = cudaMemsetAsync(grp_cnt, 0, groups * sizeof(unsigned int), s);
  if (e == cudaSuccess && groups)
    e = cudaMemsetAsync(grp_acc, 0, groups * k * 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return ht::cuda_error(e, "ht_hash_noalloc set-up copies");

  ht::KParams P;
  memset(&P, 0, sizeof P);
  for (int i = 0; i < ks->ew; ++i) P.E[i] = seed_words_host[i];
  for (int t = 0; t < ks->k; ++t)
    for (int i = 0; i < 7; ++i) P.T0[t][i] = seed_words_host[ks->off_T + t * 19 * 7 + i];
  P.seeds = reinterpret_cast<const unsigned long long *>(base + kOffSeeds);
  P.scr.grp_acc = grp_acc;
  P.scr.grp_cnt = grp_cnt;
  P.scr.str_acc = reinterpret_cast<unsigned long long *>(base + kOffStrAcc);
  P.scr.str_done = reinterpret_cast<unsigned int *>(base + kOffStrDone);
  P.scr.ctl = reinterpret_cast<ht::Ctl *>(base + kOffCtl);
  P.scr.cap_groups = max_groups;
  P.scr.cap_strings = 1;
  ht::StrPlan &sp = P.single;
  sp.ptr = static_cast<const uint8_t *>(data_dev);
  sp.len = len;
  sp.n_exec = N;
  sp.item0 = 0;
  sp.grp0 = 0;
  const uint64_t n_items = ht::items_of(N, kChunkLevels);
  sp.n_items = (uint32_t)n_items;
  P.item_begin = 0;
  P.item_end = n_items;
  P.digests = reinterpret_cast<unsigned long long *>(digest_dev);
  P.count = 1;
  const bool aligned = (reinterpret_cast<uintptr_t>(data_dev) & 15u) == 0;
  const void *func = aligned ? ks->single_aligned[kChunkLevels - 1] : ks->single_unaligned[kChunkLevels - 1];
  const int tpb = 256;
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, func, tpb, 0);
  if (e != cudaSuccess) return ht::cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (bps < 1) bps = 1;
  const uint64_t wpb = tpb / 32;
  uint64_t grid = (uint64_t)sms * (uint64_t)bps;
  const uint64_t want = (n_items + wpb - 1) / wpb;
  if (want < grid) grid = want;
  if (grid < 1) grid = 1;
  P.total_warps = (unsigned)(grid * wpb);
  void *args[] = {&P};
  e = cudaLaunchKernel(func, dim3((unsigned)grid), dim3(tpb), args, 0, s);
  if (e != cudaSuccess) return ht::cuda_error(e, "ht_hash_noalloc launch");
  return HT_OK;
}
