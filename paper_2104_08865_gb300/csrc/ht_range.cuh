// ht_range.cuh -- the hybrid kernel of the HalftimeHash hot path.
//
// The units of a launch are those of the stream kernel (one per level-1
// node, i.e. 8 executions, plus one data-less tail unit per string).  Warps
// take work items from an atomic cursor: first whole 64-execution chunks,
// where thread (x, p) hashes the eight executions of level-1 node 8c + x one
// after another with 128-bit loads (lanes 2p, 2p+1), accumulating the node in
// registers (Section 3.2 node variant, f = 8), and the eight x-threads then
// sum the level-2 node with shuffles; then, for the last stretch of the
// launch, single units, where thread x hashes execution x and level 1 is
// summed across the x-threads.  A single unit adds its level-2 term with a
// count of one to the node's accumulator (the contribution completing the
// count owns the node).  Upper levels, pending roots and the finaliser work
// as in the stream kernel.
#pragma once

#include "ht_block.cuh"
#include "ht_inc.cuh"
#include "ht_parts.cuh"
#include "ht_stream.cuh"

namespace ht {

// Ends a string segment of this warp: count its units and run the finaliser
// if they complete the string.  Every contribution of this warp to the
// string (group accumulators, pending-root sum) precedes the count.
template <int W>
__device__ __noinline__ void count_units(const KParams &P, const StrPlan &sp, unsigned s,
                                            uint64_t units, int ln) {
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0) old = atomicAdd(P.scr.str_done + s, (unsigned)units);
  old = __shfl_sync(kFull, old, 0);
  if ((uint64_t)old + units == sp.n_items) finish_string<W>(P, sp, s, ln);
}

// One round: data units [g, g_end) of string s, all inside chunk c = g >> 3.
// Thread x hashes the eight executions of level-1 node 8c + x if it is one
// of them; the round's level-2 terms are summed across the x-threads.
template <int W, bool ALIGNED>
__device__ __forceinline__ void hash_round(const KParams &P, const StrPlan &sp, unsigned s, uint64_t g,
                                           uint64_t g_end, int ln) {
  constexpr int k = Spec<W>::k;
  constexpr uint64_t B = Dims<W>::exec_bytes;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = sp.n_exec;
  const uint64_t c = g >> 3;
  const unsigned nunits = (unsigned)(g_end - g);
  const uint64_t gx = 8 * c + (uint64_t)x;
  const bool mine = gx >= g && gx < g_end;
  const int m = mine ? (int)(N - 8 * gx < 8 ? N - 8 * gx : 8) : 0;
  const uint8_t *ex = sp.ptr + 8 * gx * B + p * 16;
  const uint32_t sh = (uint32_t)(((uintptr_t)sp.ptr) & 15u);
  const bool al = ALIGNED || sh == 0;

  uint64_t n1[2][k];
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int t = 0; t < k; ++t) n1[l][t] = 0;
#pragma unroll 1
  for (int i = 0; i < m; ++i) {
    uint64_t y[2][k];
    const uint8_t *e1 = ex + i * B;
    if (kChecked && !HT_IN_RANGE(P, kChkInput, (8 * gx + i + 1) * B - 1, sp.len)) continue;
    if (al)
      ehc2_from<W>([&](int b) { return ld_stream(e1 + b * 64); }, P, y);
    else
      ehc2_from<W>([&](int b) { return ld_unaligned(e1 + b * 64, sh); }, P, y);
    if (m == 8) {
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int t = 0; t < k; ++t) n1[l][t] += (i < 7) ? nh64(y[l][t], P.T0[t][i]) : y[l][t];
    } else {
      // leaves of the incomplete last group: pending at level 0, slot i
#pragma unroll
      for (int t = 0; t < k; ++t)
        add_pending<W>(P, s, t, nh64(y[0][t], final_key<W>(P, t, 0, i, 2 * p)) +
                                    nh64(y[1][t], final_key<W>(P, t, 0, i, 2 * p + 1)));
    }
  }
  if (c < (N >> 6)) {
    // children of a level-2 node that completes: sum this round's terms
    uint64_t v0 = 0, v1 = 0;
#pragma unroll
    for (int t = 0; t < k; ++t) {
      const uint64_t key = x < 7 ? tree_key<W>(P, t, 1, x) : 0;
      uint64_t a0 = 0, a1 = 0;
      if (mine) {
        a0 = x < 7 ? nh64(n1[0][t], key) : n1[0][t];
        a1 = x < 7 ? nh64(n1[1][t], key) : n1[1][t];
      }
      a0 = x_sum(a0);
      a1 = x_sum(a1);
      if (x == t) {
        v0 = a0;
        v1 = a1;
      }
    }
    if (nunits == 8)
      push_node<W>(P, sp, s, 2, c, v0, v1, ln);
    else
      contribute_level2<W>(P, sp, s, c, v0, v1, nunits, ln);
  } else if (m == 8) {
    // complete level-1 node of the incomplete last chunk: pending, slot x
#pragma unroll
    for (int t = 0; t < k; ++t)
      add_pending<W>(P, s, t, nh64(n1[0][t], final_key<W>(P, t, 1, x, 2 * p)) +
                                  nh64(n1[1][t], final_key<W>(P, t, 1, x, 2 * p + 1)));
  }
}

// One unit that is not part of a whole-chunk item: thread x hashes execution
// 8g + x; level 1 across the x-threads; the node is either one child of a
// level-2 node that completes (count 1) or pending.
template <int W, bool ALIGNED>
__device__ __forceinline__ void hash_unit(const KParams &P, const StrPlan &sp, unsigned s, uint64_t g,
                                          int ln) {
  constexpr int k = Spec<W>::k;
  constexpr uint64_t B = Dims<W>::exec_bytes;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = sp.n_exec;
  const int m = (int)(N - 8 * g < 8 ? N - 8 * g : 8);
  const uint32_t sh = (uint32_t)(((uintptr_t)sp.ptr) & 15u);
  const uint8_t *e1 = sp.ptr + (8 * g + (uint64_t)x) * B + p * 16;
  uint64_t y[2][k];
  if (x < m && HT_IN_RANGE(P, kChkInput, (8 * g + (uint64_t)x + 1) * B - 1, sp.len)) {
    if (ALIGNED || sh == 0)
      ehc2_from<W>([&](int b) { return ld_stream(e1 + b * 64); }, P, y);
    else
      ehc2_from<W>([&](int b) { return ld_unaligned(e1 + b * 64, sh); }, P, y);
  }
  if (m < 8) {
    // leaves of the incomplete last group: pending at level 0, slot x
    if (x < m)
#pragma unroll
      for (int t = 0; t < k; ++t)
        add_pending<W>(P, s, t, nh64(y[0][t], final_key<W>(P, t, 0, x, 2 * p)) +
                                    nh64(y[1][t], final_key<W>(P, t, 0, x, 2 * p + 1)));
    return;
  }
  const uint64_t c = g >> 3;
  const int pos = (int)(g & 7);
  const bool grows = c < (N >> 6);  // the level-2 node will complete
  uint64_t v0 = 0, v1 = 0;
#pragma unroll
  for (int t = 0; t < k; ++t) {
    const uint64_t key = x < 7 ? tree_key<W>(P, t, 0, x) : 0;
    uint64_t a0 = x_sum(x < 7 ? nh64(y[0][t], key) : y[0][t]);
    uint64_t a1 = x_sum(x < 7 ? nh64(y[1][t], key) : y[1][t]);
    if (x == t) {
      if (!grows) {
        // level-1 node of the incomplete last chunk: pending, slot pos
        add_pending<W>(P, s, t, nh64(a0, final_key<W>(P, t, 1, pos, 2 * p)) +
                                    nh64(a1, final_key<W>(P, t, 1, pos, 2 * p + 1)));
      } else if (pos < 7) {
        const uint64_t k1 = tree_key<W>(P, t, 1, pos);
        v0 = nh64(a0, k1);
        v1 = nh64(a1, k1);
      } else {
        v0 = a0;
        v1 = a1;
      }
    }
  }
  if (grows) contribute_level2<W>(P, sp, s, c, v0, v1, 1, ln);
}

// ALIGNED: every string of the launch starts on a 16-byte boundary (only the
// 128-bit load path is compiled in).  A batch launch runs both variants; each
// returns at once unless the planner's alignment flag selects it.
//
// Work list, handed out by an atomic cursor: phase A, every full 64-execution
// chunk of the launch but the last nw (nw = warps in the grid), as whole
// items; phase B, every remaining unit (8 executions, or a tail unit) as its
// own item.  Warps that run ahead take more items, and the end of the launch
// is split into pieces 8 times finer than a chunk.
template <int W, bool BATCH, bool ALIGNED>
__global__ void __launch_bounds__(256, 2) range_kernel(const __grid_constant__ KParams P) {
  const int ln = threadIdx.x & 31;
  if (BATCH && (__ldcg(&P.scr.ctl->status) != 0 || (__ldcg(&P.scr.ctl->unaligned) != 0) == ALIGNED)) {
    exit_protocol(P, ln);
    return;
  }
  const uint64_t nw = P.total_warps;
  uint64_t chunks_a, units_b, b_begin = 0, c_first = 0;
  if (BATCH) {
    chunks_a = __ldcg(&P.scr.ctl->chunks_a);
    units_b = __ldcg(&P.scr.ctl->units_b);
  } else {
    // a launch over units [item_begin, item_end) of one string, item_begin
    // a chunk boundary: its whole chunks but the last nw form phase A
    c_first = P.item_begin >> 3;
    uint64_t c_last = P.item_end >> 3;
    const uint64_t C2 = P.single.n_exec >> 6;
    if (c_last > C2) c_last = C2;
    const uint64_t full = c_last > c_first ? c_last - c_first : 0;
    chunks_a = full > nw ? full - nw : 0;
    b_begin = 8 * (c_first + chunks_a);
    units_b = P.item_end - b_begin;
  }
  const uint64_t total = chunks_a + units_b;
  for (;;) {
    unsigned long long item = 0;
    if (ln == 0) item = atomicAdd(&P.scr.ctl->cursor, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    unsigned s = 0;
    uint64_t g;
    if (item < chunks_a) {
      uint64_t c;
      if (BATCH) {
        s = find_string(P.chunk0s, P.count, item);
        c = item - P.plans[s].chunk0;
      } else {
        c = c_first + item;
      }
      const StrPlan &sp = BATCH ? P.plans[s] : P.single;
      hash_round<W, ALIGNED>(P, sp, s, 8 * c, 8 * c + 8, ln);
      count_units<W>(P, sp, s, 8, ln);
      continue;
    }
    const uint64_t ub = item - chunks_a;
    if (BATCH) {
      s = find_string(P.unitb0s, P.count, ub);
      g = 8 * P.plans[s].chunks_a + (ub - P.plans[s].unitb0);
    } else {
      g = b_begin + ub;
    }
    const StrPlan &sp = BATCH ? P.plans[s] : P.single;
    if (g < ((sp.n_exec + 7) >> 3)) hash_unit<W, ALIGNED>(P, sp, s, g, ln);
    count_units<W>(P, sp, s, 1, ln);
  }
  exit_protocol(P, ln);
}

// ---- kernel tables --------------------------------------------------------------

template <int W>
KernelSet make_kernel_set() {
  KernelSet ks;
  ks.single_aligned[0] = (const void *)hash_kernel<W, 1, true, true>;
  ks.single_aligned[1] = (const void *)hash_kernel<W, 2, true, true>;
  ks.single_aligned[2] = (const void *)hash_kernel<W, 3, true, true>;
  ks.single_unaligned[0] = (const void *)hash_kernel<W, 1, true, false>;
  ks.single_unaligned[1] = (const void *)hash_kernel<W, 2, true, false>;
  ks.single_unaligned[2] = (const void *)hash_kernel<W, 3, true, false>;
  ks.batch[0] = (const void *)hash_kernel<W, 1, false, true>;
  ks.batch[1] = (const void *)hash_kernel<W, 2, false, true>;
  ks.batch[2] = (const void *)hash_kernel<W, 3, false, true>;
  ks.batch_unaligned[0] = (const void *)hash_kernel<W, 1, false, false>;
  ks.batch_unaligned[1] = (const void *)hash_kernel<W, 2, false, false>;
  ks.batch_unaligned[2] = (const void *)hash_kernel<W, 3, false, false>;
  ks.batch_map[0] = nullptr;
  ks.batch_map[1] = (const void *)hash_kernel<W, 2, false, true, false, kLanes, true>;
  ks.batch_map[2] = (const void *)hash_kernel<W, 3, false, true, false, kLanes, true>;
  ks.batch_unaligned_map[0] = nullptr;
  ks.batch_unaligned_map[1] = (const void *)hash_kernel<W, 2, false, false, false, kLanes, true>;
  ks.batch_unaligned_map[2] = (const void *)hash_kernel<W, 3, false, false, false, kLanes, true>;
  ks.plan[0] = (const void *)plan_kernel<W, 0>;
  ks.plan[1] = (const void *)plan_kernel<W, 1>;
  ks.plan[2] = (const void *)plan_kernel<W, 2>;
  ks.plan[3] = (const void *)plan_kernel<W, 3>;
  ks.plan_tiles[0] = (const void *)plan_tiles_kernel<W, 0>;
  ks.plan_tiles[1] = (const void *)plan_tiles_kernel<W, 1>;
  ks.plan_tiles[2] = (const void *)plan_tiles_kernel<W, 2>;
  ks.plan_tiles[3] = (const void *)plan_tiles_kernel<W, 3>;
  ks.plan_totals = (const void *)plan_totals_kernel<W>;
  ks.plan_items = (const void *)plan_items_kernel<W>;
  ks.plan_write[0] = (const void *)plan_write_kernel<W, 0>;
  ks.plan_write[1] = (const void *)plan_write_kernel<W, 1>;
  ks.plan_write[2] = (const void *)plan_write_kernel<W, 2>;
  ks.plan_write[3] = (const void *)plan_write_kernel<W, 3>;
  ks.stream_single = (const void *)stream_kernel<W, false>;
  ks.stream_batch = (const void *)stream_kernel<W, true>;
  ks.block_single = (const void *)block_kernel<W, true>;
  ks.block_single_unaligned = (const void *)block_kernel<W, false>;
  ks.range_single = (const void *)range_kernel<W, false, true>;
  ks.range_single_unaligned = (const void *)range_kernel<W, false, false>;
  ks.range_batch = (const void *)range_kernel<W, true, true>;
  ks.range_batch_unaligned = (const void *)range_kernel<W, true, false>;
  ks.part_tail = (const void *)part_tail_kernel<W>;
  ks.part_finish = (const void *)part_finish_kernel<W, 2>;
  ks.inc_aligned = (const void *)hash_kernel<W, 2, true, true, true>;
  ks.inc_unaligned = (const void *)hash_kernel<W, 2, true, false, true>;
  ks.inc_block_aligned = (const void *)block_kernel<W, true, true>;
  ks.inc_block_unaligned = (const void *)block_kernel<W, false, true>;
  ks.inc_stack = (const void *)inc_stack_kernel<W>;
  ks.wait_probe = (const void *)wait_probe_kernel<W>;
  ks.exec_bytes = Dims<W>::exec_bytes;
  ks.k = Spec<W>::k;
  ks.n_seed = Dims<W>::n_seed;
  ks.off_T = Dims<W>::off_T;
  ks.off_F = Dims<W>::off_F;
  ks.off_R = Dims<W>::off_R;
  ks.ew = Dims<W>::ew;
  ks.lanes = kLanes;
  ks.tree = 0;
  return ks;
}

}  // namespace ht
