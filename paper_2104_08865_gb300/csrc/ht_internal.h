// ht_internal.h -- structures shared by the host runtime and the kernels of
// libhalftime (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ht {

// One string of a launch, as the planner lays it out.  In incremental mode
// (one update of whole 64-execution chunks) chunk0 is the number of chunks
// the string held before the update and n_exec counts the executions up to
// the update's end.
struct StrPlan {
  const uint8_t *ptr;  // first byte of the string (device)
  uint64_t len;        // bytes
  uint64_t n_exec;     // N = floor(len / exec_bytes): EHC executions
  uint64_t item0;      // first global work item of this string
  uint64_t grp0;       // first tree-group slot of this string in scratch
  uint32_t n_items;    // work items: max(1, ceil(N / 8^L)), or stream/range units
  uint32_t pad;
  // hybrid kernel work list (planner): full 64-execution chunks before this
  // string in the batch, full chunks of this string taken whole in phase A,
  // and phase-B units before this string
  uint64_t chunk0;
  uint64_t chunks_a;
  uint64_t unitb0;
};

// Launch-wide control words (one per context).  cursor and exit return to 0
// at the end of every hash launch; status is sticky until the host reads it.
struct Ctl {
  unsigned long long cursor;  // next work item to hand out
  unsigned long long total;   // work items of the current batch (planner)
  unsigned long long groups;  // tree-group slots the batch needs (planner)
  unsigned long long chunks_a;  // hybrid kernel: phase-A work items (whole chunks)
  unsigned long long units_b;   // hybrid kernel: phase-B work items (single units)
  unsigned int exit;          // warps that have left the work loop
  unsigned int status;        // 0 or kStatus* bits
  unsigned int unaligned;     // planner: some string of the batch is not 16-byte aligned
  unsigned int bad_kind;      // checked build: kind of the first out-of-range access (0: none)
  unsigned long long bad_index;  // checked build: its index
};
constexpr unsigned int kStatusTooLong = 1;  // a batch exceeded the scratch
// (kStatusTimeout = 2: a bounded wait on a stage's mbarrier ran out;
//  kStatusBounds = 4: the checked build skipped an out-of-range access)

// Device scratch of one context.
struct Scratch {
  unsigned long long *grp_acc;  // [cap_groups][k][8] node accumulators
  unsigned int *grp_cnt;        // [cap_groups] arrivals per group
  unsigned long long *str_acc;  // [cap_strings][k] pending-root sums
  unsigned int *str_done;       // [cap_strings] finished items per string
  Ctl *ctl;
  uint64_t cap_groups;
  uint64_t cap_strings;
};

// Kernel parameters (passed as a __grid_constant__ struct: the hash keys of
// the EHC step become constant-bank operands of the integer instructions).
struct KParams {
  unsigned long long E[30];     // EHC hash keys, e*w words
  unsigned long long T0[5][8];  // level-0 tree keys per tree (7 used)
  const unsigned long long *seeds;  // all seed words on the device
  Scratch scr;
  const StrPlan *plans;         // batch mode: planner output
  const unsigned long long *item0s;  // batch mode: item0 of each string (+ total)
  const unsigned long long *chunk0s;  // batch mode: chunk0 of each string (+ total)
  const unsigned long long *unitb0s;  // batch mode: unitb0 of each string (+ total)
  const unsigned int *item_str;  // batch mode: the string of every work item (or null: search item0s)
  unsigned long long *digests;  // count * k words
  unsigned long long *stack;    // incremental mode: pending nodes [level][8][k][8] (written)
  const unsigned long long *stack_in;  // incremental mode: the previous update's stack (read)
  const uint8_t *inc_first;     // incremental mode: bytes of chunk chunk0 if not at ptr (else null)
  unsigned long long inc_fill;  // block-chunk update: only this many bytes of it are at inc_first
  unsigned long long inc_stage_src;  // ... and the rest start the update, at this address
  unsigned long long inc_chunk0_slot;  // warp-chunk update with inc_fill: the first chunk's group slot
  // incremental mode: the bytes after the update's last whole chunk, which
  // the kernel copies into the handle's other buffer for the next update
  const uint8_t *inc_rem_src;
  uint8_t *inc_rem_dst;
  unsigned long long inc_rem_len;
  StrPlan single;               // single-string mode: the string
  unsigned long long item_begin, item_end;  // single mode: item range of this launch
  unsigned int count;           // batch mode: strings
  unsigned int total_warps;     // warps in the grid
  unsigned int stages;          // stream kernel: shared-memory slots per warp
  long long wait_cycles;        // stream kernel: limit of a stage wait (0: the default, about 1 s)
};

struct PlanArgs {
  const void *const *ptrs;
  const uint64_t *lens;
  unsigned int count;
  StrPlan *plans;
  unsigned long long *item0s;
  unsigned long long *chunk0s;
  unsigned long long *unitb0s;
  Ctl *ctl;
  uint64_t cap_groups;
  unsigned int total_warps;  // warps of the hash kernel (hybrid work list)
  // multi-block planner: per tile of 1024 strings, its item and group totals
  // (then their exclusive prefix sums) and whether it holds an unaligned string
  unsigned long long *tile_items;
  unsigned long long *tile_groups;
  unsigned int *tile_flags;
  unsigned int n_tiles;
  // warp-chunk batches: the string of every work item (capacity cap_items;
  // 0 when the batch kernel searches item0s instead)
  unsigned int *item_str;
  uint64_t cap_items;
};

// Kernel variants of one width.  Warp-chunk kernels: chunk height L in
// {1, 2, 3}; single-string or batch; batch kernels also carry the
// unaligned-load path.  Stream kernels (TMA stages): single-string or batch.
// Planners: [0] stream units, [L] warp-chunk items of height L.
struct KernelSet {
  const void *single_aligned[3];    // [L-1]
  const void *single_unaligned[3];  // [L-1]
  const void *batch[3];             // [L-1], aligned-only
  const void *batch_unaligned[3];   // [L-1], general (see ctl.unaligned)
  const void *batch_map[3];         // [L-1], L >= 2: the same, strings found through the item map
  const void *batch_unaligned_map[3];
  const void *plan[4];              // [0]: stream, [L]: warp-chunk (one block, hybrid work list too)
  const void *plan_tiles[4];        // multi-block planner, same index: tile totals
  const void *plan_totals;          //   their prefix sums and the batch totals
  const void *plan_write[4];        //   every string's plan
  const void *plan_items;           //   the string of every work item
  const void *stream_single;
  const void *stream_batch;
  const void *block_single;  // block-chunk kernel: a block of 8 warps per 64-execution chunk
  const void *block_single_unaligned;
  const void *range_single;  // hybrid kernel: chunks then units from a cursor
  const void *range_single_unaligned;
  const void *range_batch;   // [aligned-only, general] pair, see ctl.unaligned
  const void *range_batch_unaligned;
  const void *part_tail;    // parts: tail NH of the last part
  const void *part_finish;  // parts: climb merged groups, write the digest
  const void *inc_aligned;    // incremental: whole chunks of one update
  const void *inc_unaligned;
  const void *inc_block_aligned;    // the same with the block-chunk kernel (short updates)
  const void *inc_block_unaligned;
  const void *inc_stack;      // incremental: pending stack nodes into the sum
  const void *wait_probe;     // a bounded wait that runs out (tests the timeout path)
  int exec_bytes, k, n_seed, off_T, off_F, off_R, ew;
  // words per block: 8, or 4 for the 256-bit-block variant, whose set holds
  // only the warp-chunk kernels with 64-execution sub-chunks (index L = 2)
  // and the multi-block planner; its other entries are null
  int lanes;
  // tree: 0 for the paper's T-hat (8-ary, pending roots, final NH), 1 for the
  // binary-tree ablation (Eq. algebraic-badger over all EHC outputs; its set
  // holds the single and batch kernels with 64-execution items (index L = 2)
  // and the multi-block planner; level keys at off_T + 64 t + h)
  int tree;
};

const KernelSet &kernels_w16();
const KernelSet &kernels_w24();
const KernelSet &kernels_w32();
const KernelSet &kernels_w40();
// the same widths with 256-bit blocks
const KernelSet &kernels_w16_v3();
const KernelSet &kernels_w24_v3();
const KernelSet &kernels_w32_v3();
const KernelSet &kernels_w40_v3();
// the same widths under the binary-tree ablation
const KernelSet &kernels_w16_bin();
const KernelSet &kernels_w24_bin();
const KernelSet &kernels_w32_bin();
const KernelSet &kernels_w40_bin();

}  // namespace ht
