// ht_badger.cuh -- the binary-tree ablation of HalftimeHash for sm_103a: the
// approach of Badger that the paper's tree T-hat improves on (Section 5.2,
// closing paragraph), built so that the two can be measured side by side.
//
// Per tree t the EHC outputs of every execution and lane form one sequence,
// execution-major and lane-minor (leaf 8x + lane), and Carter and Wegman's
// tree T (Eq. algebraic-badger, Section 3.1) consumes it whole: a span of
// n > 1 leaves splits after its first 2^(ceil(lg n) - 1) leaves, and the
// fan-out-2 node of Section 3.2, H(k_i, left, right) = NH(left, k_i) + right,
// joins the halves with i = ceil(lg n) - 1.  There are no pending roots and
// no final NH; the Toeplitz tail with the length word is added as usual.
//
// Unrolled, T of n leaves is the sum over the complete subtrees that the
// binary digits of n cut the sequence into (largest first): each enters as
// NH(root, k_h), h its height, except the last one, which enters unhashed.
// With 8 lanes the digits of 8N are those of N shifted by three, so every
// complete subtree of height >= 3 covers whole executions, and:
//   * within one execution (heights 1..3): lanes 2p, 2p+1 in thread (x, p),
//     then shuffles across p;
//   * within a 64-execution work item (heights 4..6 over the eight
//     executions 8x .. 8x+7 of thread (x, p), in registers; heights 7..9 by
//     shuffles across x): the item's root, of height 9;
//   * above the item: the binary tree across warps, with the same
//     order-free protocol as the default kernels at fan-out 2 (the left child
//     adds NH(v, k_h) into its parent's accumulator, the right child v; the
//     second arrival takes the parent and climbs on).
// The last node of an odd count at its height is a complete subtree of the
// digit decomposition: its term goes straight into the string's sum.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

// Key k_h of tree t above height 7 (heights 0..7 travel in KParams.T0).
template <int W>
__device__ __forceinline__ uint64_t bin_key(const KParams &P, int t, int h) {
  const int r = t * kBinLevels + h;
  if (!HT_IN_RANGE(P, kChkSeedT, r, Spec<W>::k * kBinLevels)) return 0;
  return __ldg(P.seeds + BinDims<W>::off_T + r);
}

// The fan-out-2 tree node: the left child through NH under key, the right
// child as is (Section 3.2 variant).
__device__ __forceinline__ uint64_t bnode(uint64_t left, uint64_t right, uint64_t key) {
  return nh64(left, key) + right;
}

// Joins this thread's node with its partner across lane bit `bit` (lane ^
// (1 << bit)): the thread whose bit is clear holds the left child.
__device__ __forceinline__ uint64_t bjoin(uint64_t v, unsigned mask, int ln, int bit, uint64_t key) {
  const uint64_t o = __shfl_xor_sync(mask, v, 1 << bit);
  return ((ln >> bit) & 1) ? bnode(o, v, key) : bnode(v, o, key);
}

// A complete subtree of height h that the digit decomposition leaves whole:
// its term in the string's sum (the lowest such subtree, height hmin, enters
// unhashed).
template <int W>
__device__ __forceinline__ uint64_t bin_term(const KParams &P, int t, int h, int hmin, uint64_t v) {
  if (h == hmin) return v;
  return nh64(v, h < 8 ? P.T0[t][h] : bin_key<W>(P, t, h));
}

// Trees a thread carries above an execution: after the lanes are joined all
// four p-threads hold the same node values, so thread (x, p) keeps trees
// p and p + 4 only (kOwn of them), which keeps the binary counter small.
template <int W>
struct BinOwn {
  static constexpr int n = (Spec<W>::k + 3) / 4;
};

// Levels 0..9 of work item c (64 executions) of a string whose bytes start at
// base.  A full item's root (height 9) is returned in root[j] = tree p + 4j
// of every lane (x, p) with p + 4j < k; in the string's last, incomplete
// item the complete subtrees of the digit decomposition add their terms to
// pend.  Returns whether the item is full.  Touches no scratch.
template <int W, bool ALIGNED>
__device__ __forceinline__ bool bin_item_root(const KParams &P, const StrPlan &sp, const uint8_t *base,
                                              uint64_t c, int ln, uint64_t (&pend)[Spec<W>::k],
                                              bool &anyp, uint64_t (&root)[BinOwn<W>::n]) {
  constexpr int k = Spec<W>::k, KO = BinOwn<W>::n;
  constexpr uint64_t XB = Dims<W>::exec_bytes;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = sp.n_exec;
  const uint64_t e0 = c * 64;
  if (e0 >= N) return false;
  const uint32_t sh = ALIGNED ? 0u : (uint32_t)(((uintptr_t)base) & 15u);
  const int m = (int)((N - e0) < 64 ? (N - e0) : 64);
  int cnt = m - 8 * x;
  cnt = cnt < 0 ? 0 : (cnt > 8 ? 8 : cnt);
  const unsigned gmask = 0xFu << (4 * x);  // the four p-threads of execution group x
  const uint8_t *ex = base + (e0 + 8ull * x) * XB;
  // key of height 3 + h of owned tree j
  auto K = [&](int j, int h) -> uint64_t {
    uint64_t v = 0;
#pragma unroll
    for (int t = 0; t < k; ++t)
      if (t == p + 4 * j) v = P.T0[t][3 + h];
    return v;
  };
  // binary counter over this thread's executions, owned trees: pending
  // nodes of heights 3, 4, 5, and the height-6 node of all eight
  uint64_t a3[KO], a4[KO], a5[KO], n6[KO];
#pragma unroll
  for (int j = 0; j < KO; ++j) a3[j] = a4[j] = a5[j] = n6[j] = 0;
  auto step = [&](int s) {
    uint64_t y[2][k];
    ehc2<W, ALIGNED>(ex + s * XB, p, sh, P, y);
    uint64_t e[k];
#pragma unroll
    for (int t = 0; t < k; ++t) {
      // heights 1..3: the execution's eight lanes
      e[t] = bnode(y[0][t], y[1][t], P.T0[t][0]);
      e[t] = bjoin(e[t], gmask, ln, 0, P.T0[t][1]);
      e[t] = bjoin(e[t], gmask, ln, 1, P.T0[t][2]);
    }
#pragma unroll
    for (int j = 0; j < KO; ++j) {
      uint64_t ej = 0;
#pragma unroll
      for (int t = 0; t < k; ++t)
        if (t == p + 4 * j) ej = e[t];
      // heights 4..6: the thread's executions, as a binary counter
      if ((s & 1) == 0) {
        a3[j] = ej;
      } else {
        const uint64_t n4 = bnode(a3[j], ej, K(j, 0));
        if ((s & 2) == 0) {
          a4[j] = n4;
        } else {
          const uint64_t n5 = bnode(a4[j], n4, K(j, 1));
          if ((s & 4) == 0) a5[j] = n5;
          else n6[j] = bnode(a5[j], n5, K(j, 2));
        }
      }
    }
  };
  if (m == 64) {
    // (one execution per iteration: two would spill with the counter)
#pragma unroll 1
    for (int s = 0; s < 8; ++s) {
      if (kChecked && !HT_IN_RANGE(P, kChkInput, (e0 + 8ull * x + s + 1) * XB - 1, sp.len)) continue;
      step(s);
    }
  } else {
#pragma unroll 1
    for (int s = 0; s < cnt; ++s) {
      if (kChecked && !HT_IN_RANGE(P, kChkInput, (e0 + 8ull * x + s + 1) * XB - 1, sp.len)) continue;
      step(s);
    }
  }
  // heights 7..9 across the eight execution groups
  const int hmin = 3 + (__ffsll((long long)N) - 1);
  const int G = m >> 3;  // execution groups with all eight executions
#pragma unroll
  for (int j = 0; j < KO; ++j) {
    const int t = p + 4 * j;  // (>= k: a lane with nothing to keep)
    const uint64_t n7 = bjoin(n6[j], kFull, ln, 2, K(j, 3));
    const uint64_t n8 = bjoin(n7, kFull, ln, 3, K(j, 4));
    if (m == 64) {
      root[j] = bjoin(n8, kFull, ln, 4, t < k ? bin_key<W>(P, t, 8) : 0);
    } else if (t < k) {
      // the digit decomposition of the item's m executions: groups of
      // 32, 16, 8 executions (bits 2..0 of G), then 4, 2, 1 executions of
      // group G (bits 2..0 of m & 7)
      uint64_t add = 0;
      if ((G & 4) && x == 0) add += bin_term<W>(P, t, 8, hmin, n8);
      if ((G & 2) && x == (G & 4)) add += bin_term<W>(P, t, 7, hmin, n7);
      if ((G & 1) && x == G - 1) add += bin_term<W>(P, t, 6, hmin, n6[j]);
      if (x == G) {
        if (cnt & 4) add += bin_term<W>(P, t, 5, hmin, a5[j]);
        if (cnt & 2) add += bin_term<W>(P, t, 4, hmin, a4[j]);
        if (cnt & 1) add += bin_term<W>(P, t, 3, hmin, a3[j]);
      }
#pragma unroll
      for (int u = 0; u < k; ++u)
        if (u == t) pend[u] += add;
    }
  }
  if (m < 64) anyp = true;
  return m == 64;
}

// Carries node idx of height 9 (the root of full item idx) up the binary tree
// across warps: as long as this warp's arrival completes a pair, it takes the
// parent and goes on one height up.  Thread t < k adds tree t's values.
// Group slots: heights from 9 up, C_h >> 1 pairs at height h, where
// C_h = N >> (h - 3); accumulators are k words per slot.
template <int W>
__device__ void bin_climb(const KParams &P, const StrPlan &sp, uint64_t idx, const uint64_t (&root)[BinOwn<W>::n],
                          int ln, uint64_t (&pend)[Spec<W>::k], bool &anyp) {
  constexpr int k = Spec<W>::k, KO = BinOwn<W>::n;
  const uint64_t N = sp.n_exec;
  const int hmin = 3 + (__ffsll((long long)N) - 1);
  uint64_t goff = 0;
  // tree ln's value in lane ln < k (lane ln = (x, p) holds tree p + 4 (ln >> 2))
  uint64_t mine = 0;
#pragma unroll
  for (int j = 0; j < KO; ++j)
    if ((ln >> 2) == j) mine = root[j];
  for (int h = 9;; ++h) {
    const uint64_t C = N >> (h - 3);
    if (idx >= (C & ~1ull)) {
      // the last node of an odd count: a complete subtree of the digit
      // decomposition
#pragma unroll
      for (int t = 0; t < k; ++t)
        if (ln == t) pend[t] += bin_term<W>(P, t, h, hmin, mine);
      anyp = true;
      return;
    }
    const uint64_t slot = sp.grp0 + goff + (idx >> 1);
    const bool ok = HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups);
    if (ln < k && ok) {
      const uint64_t a = (idx & 1) ? mine : nh64(mine, bin_key<W>(P, ln, h));
      atomicAdd(P.scr.grp_acc + slot * k + (uint64_t)ln, (unsigned long long)a);
    }
    if (arrive(P, slot, ln) != 2) return;
    __threadfence();
    if (ln < k && ok) {
      unsigned long long *acc = P.scr.grp_acc + slot * k + (uint64_t)ln;
      mine = ld_cg(acc);
      *acc = 0;
    }
    if (ln == 0 && ok) P.scr.grp_cnt[slot] = 0;
    goff += C >> 1;
    idx >>= 1;
  }
}

// One work item of a batch under the binary-tree ablation: its levels, the
// climb, and the string's completion count.
template <int W, bool ALIGNED>
__device__ void bin_chunk(const KParams &P, const StrPlan &sp, unsigned sidx, uint64_t c, int ln) {
  constexpr int k = Spec<W>::k;
  uint64_t pend[k], root[BinOwn<W>::n];
#pragma unroll
  for (int t = 0; t < k; ++t) pend[t] = 0;
  bool anyp = false;
  const bool full = bin_item_root<W, ALIGNED>(P, sp, sp.ptr, c, ln, pend, anyp, root);
  if (full) bin_climb<W>(P, sp, c, root, ln, pend, anyp);
  if (sp.n_items == 1) {
    finish_local<W, kLanes, true>(P, sp, sidx, pend, ln);
    return;
  }
  flush_pending<W>(P, sidx, pend, anyp, ln);
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0 && HT_IN_RANGE(P, kChkString, sidx, P.scr.cap_strings)) old = atomicAdd(P.scr.str_done + sidx, 1u);
  old = __shfl_sync(kFull, old, 0);
  if (old == sp.n_items - 1) finish_string<W, kLanes, true>(P, sp, sidx, ln);
}

// The binary-tree ablation's kernel: single strings (items from the cursor;
// the last warp to leave writes the digest) or batches (planner output, an
// aligned-only and a general instance as for the default kernels).
template <int W, bool SINGLE, bool ALIGNED>
__global__ void __launch_bounds__(256, 2) bin_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  const int ln = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if constexpr (SINGLE) {
    // (launched to overlap its predecessor, it waits for it here: no part of
    // this kernel is arranged to run before the scratch is free)
    griddep_wait();
    const StrPlan &sp = P.single;
    bool first = true;
    for (;;) {
      unsigned long long item = 0;
      if (first) {
        item = P.item_begin + gw;
        first = false;
      } else {
        if (P.item_end - P.item_begin <= P.total_warps) break;
        if (ln == 0) item = atomicAdd(&P.scr.ctl->cursor, 1ull);
        item = __shfl_sync(kFull, item, 0) + P.item_begin + P.total_warps;
      }
      if (item >= P.item_end) break;
      uint64_t pend[k], root[BinOwn<W>::n];
#pragma unroll
      for (int t = 0; t < k; ++t) pend[t] = 0;
      bool anyp = false;
      const bool full = bin_item_root<W, ALIGNED>(P, sp, sp.ptr, item, ln, pend, anyp, root);
      if (full) bin_climb<W>(P, sp, item, root, ln, pend, anyp);
      flush_pending<W>(P, 0, pend, anyp, ln);
    }
    const bool last = exit_protocol(P, ln);
    if (last && P.item_end >= P.single.n_items) finish_string<W, kLanes, true>(P, P.single, 0, ln);
  } else {
    if (__ldcg(&P.scr.ctl->status) != 0 || (__ldcg(&P.scr.ctl->unaligned) != 0) == ALIGNED) {
      exit_protocol(P, ln);
      return;
    }
    const uint64_t total = __ldcg(&P.scr.ctl->total);
    for (;;) {
      unsigned long long item = 0;
      if (ln == 0) item = atomicAdd(&P.scr.ctl->cursor, 1ull);
      item = __shfl_sync(kFull, item, 0);
      if (item >= total) break;
      const unsigned s = find_string_warp(P.item0s, P.count, item, ln);
      const StrPlan sp = P.plans[s];
      const uint64_t c = item - sp.item0;
      if (ALIGNED || (((uintptr_t)sp.ptr) & 15u) == 0)
        bin_chunk<W, true>(P, sp, s, c, ln);
      else
        bin_chunk<W, false>(P, sp, s, c, ln);
    }
    exit_protocol(P, ln);
  }
}

// Kernel table of the binary-tree ablation: the kernels above with
// 64-execution work items (index L = 2) and the multi-block planner counting
// the ablation's group slots.
template <int W>
inline KernelSet make_kernel_set_bin() {
  constexpr int L = 2;
  KernelSet ks = {};
  ks.single_aligned[L - 1] = (const void *)bin_kernel<W, true, true>;
  ks.single_unaligned[L - 1] = (const void *)bin_kernel<W, true, false>;
  ks.batch[L - 1] = (const void *)bin_kernel<W, false, true>;
  ks.batch_unaligned[L - 1] = (const void *)bin_kernel<W, false, false>;
  ks.plan_tiles[L] = (const void *)plan_tiles_kernel<W, L, kLanes, true>;
  ks.plan_totals = (const void *)plan_totals_kernel<W>;
  ks.plan_items = (const void *)plan_items_kernel<W>;
  ks.plan_write[L] = (const void *)plan_write_kernel<W, L, kLanes, true>;
  ks.exec_bytes = Dims<W>::exec_bytes;
  ks.k = Spec<W>::k;
  ks.n_seed = BinDims<W>::n_seed;
  ks.off_T = BinDims<W>::off_T;
  ks.off_F = BinDims<W>::off_R;  // (no final-NH region)
  ks.off_R = BinDims<W>::off_R;
  ks.ew = Dims<W>::ew;
  ks.lanes = kLanes;
  ks.tree = 1;
  return ks;
}

}  // namespace ht
