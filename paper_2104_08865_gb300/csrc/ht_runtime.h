// ht_runtime.h -- host-side state of a libhalftime context (internal).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

#include "halftime.h"
#include "ht_internal.h"

constexpr int kStageSlots = 4;  // staging ring of ht_hash_host

struct ht_ctx {
  int width = 0;
  int device = 0;
  int num_sms = 1;
  int smem_optin = 0;  // max dynamic shared memory per block
  unsigned flags = 0;  // HT_FLAG_*
  const ht::KernelSet *ks = nullptr;
  std::vector<uint64_t> h_seeds;
  unsigned long long *d_seeds = nullptr;
  uint64_t *d_digest = nullptr;  // k words, for host-side calls
  // scratch (see ht::Scratch)
  unsigned long long *grp_acc = nullptr;
  unsigned int *grp_cnt = nullptr;
  unsigned long long *str_acc = nullptr;
  unsigned int *str_done = nullptr;
  ht::StrPlan *plans = nullptr;
  unsigned long long *item0s = nullptr;
  unsigned long long *chunk0s = nullptr;
  unsigned long long *unitb0s = nullptr;
  unsigned long long *tile_items = nullptr;   // multi-block planner, per 1024 strings
  unsigned long long *tile_groups = nullptr;
  unsigned int *tile_flags = nullptr;
  unsigned int *item_str = nullptr;  // warp-chunk batches: the string of every work item
  uint64_t cap_items = 0;
  ht::Ctl *ctl = nullptr;
  uint64_t cap_groups = 0, cap_strings = 0;
  // launch shapes: [0..63] by floor(log2(len)), [64] batches
  ht_shape shapes[65];
  // batch graphs (planner -> persistent kernel): [0] for batches of up to
  // 1024 strings, planned by one block, [1] for the others
  struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node_plan = nullptr, node_hash = nullptr, node_hash2 = nullptr;
    cudaGraphNode_t node_totals = nullptr, node_write = nullptr;  // multi-block planner (else null)
    cudaGraphNode_t node_items = nullptr;  // item -> string map (warp-chunk kernel, L >= 2; else null)
    ht_shape shape = {};
    bool map = false;  // the planner writes the item map and the kernels read it
    bool valid = false;
  } graphs[2];
  ht::PlanArgs plan_args = {};
  ht::KParams batch_params = {};
  // host-input pipeline
  cudaStream_t copy_stream = nullptr;
  uint8_t *stage[kStageSlots] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t stage_bytes = 0;
  cudaEvent_t ev_copy[kStageSlots] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_hash[kStageSlots] = {nullptr, nullptr, nullptr, nullptr};
  // one string in parts (ht_part_*)
  unsigned long long *part_buf = nullptr;
  uint64_t part_cap_words = 0, part_len = 0;
  bool part_open = false;
  bool part_owned = false;  // part_buf allocated by the library
  std::atomic<uint64_t> launches{0};
  long long wait_cycles = 0;  // testing: limit of the stream kernel's stage waits (0: default)
  // blocks per SM of (kernel, threads per block, dynamic shared memory),
  // queried once per context (the query costs more than a small launch)
  struct Occ {
    const void *func;
    int tpb;
    size_t smem;
    int blocks;
  };
  std::vector<Occ> occ_cache;
};

namespace ht {
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
const KernelSet *kernel_set(int width);
// Work items of a string of N executions for the warp-chunk kernel with
// chunk height L and blocks of `lanes` words (8 or 4; at least one item).
uint64_t items_of(uint64_t N, int L, int lanes = 8);
uint64_t groups_of(uint64_t N, int L);
// The next output of splitmix64 (Steele, Lea and Flood 2014) from *state.
uint64_t splitmix64_next(uint64_t *state);
// Zeroes P, then fills the hash keys, the seed pointer and the context's scratch.
void fill_keys(const ht_ctx *c, KParams &P);
// Waits for the stream, then reads and clears a control block's status word;
// returns HT_OK or the error it reports.
int read_status(Ctl *ctl, cudaStream_t s);
}  // namespace ht
