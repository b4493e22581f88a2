// ht_inc.cuh -- kernels of incremental hashing (init / update / final).
//
// An update hashes whole 64-execution chunks, the level-2 nodes of the
// string's trees (Section 5.2), in the string's global chunk frame.  Between
// updates the trees' eager counter is carried on a stack: for every level
// l >= 2 the nodes of the last, incomplete group, which are the pending nodes
// of a string that ends here, one value per tree and lane.  While a later
// update completes that group, the group's accumulator has to start from
// these nodes (inc_seed_kernel); when the string ends they are hashed with
// their final keys like any other pending node (inc_stack_kernel).  Bytes
// that do not fill a chunk wait in a buffer; the final launch hashes them
// (fewer than 64 executions: the level-0 and level-1 pending nodes) and the
// tail, so the digest equals the one-shot digest of the whole string.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

__device__ __forceinline__ unsigned long long *stack_node(const KParams &P, int k, int lvl, uint64_t j,
                                                          int t, int lane) {
  return P.stack + (((uint64_t)lvl * kFan + j) * k + (uint64_t)t) * kLanes + lane;
}

// Before an update of chunks [chunk0, n_exec / 64): every level whose
// incomplete group (d > 0 nodes on the stack) is completed by the update gets
// that group's accumulator and arrival count from the stack nodes, in the
// group slot that the update kernel uses for it (the first slot of the
// level).  One warp; thread (x, p) handles tree x, lanes 2p and 2p+1.
template <int W>
__global__ void __launch_bounds__(32) inc_seed_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  const int ln = threadIdx.x & 31;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N0 = P.single.chunk0 << 6, N1 = P.single.n_exec;
  uint64_t goff = 0;
  for (int lvl = 2; lvl < kLevels - 1; ++lvl) {
    const uint64_t n0 = N0 >> (3 * lvl), n1 = N1 >> (3 * lvl);
    const uint64_t gbase = n0 >> 3, gend = n1 >> 3;  // groups the update completes
    const int d = (int)(n0 & 7);
    if (gend > gbase && d > 0) {
      if (x < k) {
        uint64_t a0 = 0, a1 = 0;
        for (int j = 0; j < d; ++j) {  // j < 7: every stack node is hashed
          const uint64_t key = tree_key<W>(P, x, lvl, j);
          a0 += nh64(*stack_node(P, k, lvl, j, x, 2 * p), key);
          a1 += nh64(*stack_node(P, k, lvl, j, x, 2 * p + 1), key);
        }
        unsigned long long *acc = P.scr.grp_acc + (goff * k + (uint64_t)x) * kLanes + 2 * p;
        acc[0] = a0;
        acc[1] = a1;
      }
      if (ln == 0) P.scr.grp_cnt[goff] = (unsigned)d;
    }
    goff += gend - gbase;
  }
}

// At the end of the string (n_exec executions in all): the pending nodes of
// levels >= 2 are the stack's (digit l of n_exec in base 8 at level l);
// their final NH (Section 6.1) goes into the string's sum.  One warp.
template <int W>
__global__ void __launch_bounds__(32) inc_stack_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  const int ln = threadIdx.x & 31;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = P.single.n_exec;
  uint64_t s = 0;
  if (x < k) {
    for (int lvl = 2; lvl < kLevels; ++lvl) {
      const int d = (int)((N >> (3 * lvl)) & 7);
      for (int j = 0; j < d; ++j)
        s += nh64(*stack_node(P, k, lvl, j, x, 2 * p), final_key<W>(P, x, lvl, j, 2 * p)) +
             nh64(*stack_node(P, k, lvl, j, x, 2 * p + 1), final_key<W>(P, x, lvl, j, 2 * p + 1));
    }
  }
  s += __shfl_xor_sync(kFull, s, 1);
  s += __shfl_xor_sync(kFull, s, 2);
  if (x < k && p == 0) atomicAdd(P.scr.str_acc + x, (unsigned long long)s);
}

}  // namespace ht
