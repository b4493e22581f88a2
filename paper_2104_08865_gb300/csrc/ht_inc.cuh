// ht_inc.cuh -- kernels of incremental hashing (init / update / final).
//
// An update hashes whole 64-execution chunks, the level-2 nodes of the
// string's trees (Section 5.2), in the string's global chunk frame, with the
// block-chunk or the warp-chunk kernel in its incremental mode (a block or a
// warp of its own also starts the groups that the update completes from the
// stack: seed_frontier).  Between
// updates the trees' eager counter is carried on a stack: for every level
// l >= 2 the nodes of the last, incomplete group, which are the pending nodes
// of a string that ends here, one value per tree and lane.  When the string
// ends they are hashed with their final keys like any other pending node
// (inc_stack_kernel).  Bytes that do not fill a chunk wait in a buffer; the
// final launch hashes them (fewer than 64 executions: the level-0 and
// level-1 pending nodes) and the tail, so the digest equals the one-shot
// digest of the whole string.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

__device__ __forceinline__ unsigned long long *stack_node(const KParams &P, int k, int lvl, uint64_t j,
                                                          int t, int lane) {
  return P.stack + (((uint64_t)lvl * kFan + j) * k + (uint64_t)t) * kLanes + lane;
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
      for (int j = 0; j < d; ++j) {
        const uint64_t o = (((uint64_t)lvl * kFan + j) * k + (uint64_t)x) * kLanes + 2 * p;
        if (!HT_IN_RANGE(P, kChkStack, o + 1, (uint64_t)kLevels * kFan * k * kLanes)) continue;
        (void)o;
        s += nh64(*stack_node(P, k, lvl, j, x, 2 * p), final_key<W>(P, x, lvl, j, 2 * p)) +
             nh64(*stack_node(P, k, lvl, j, x, 2 * p + 1), final_key<W>(P, x, lvl, j, 2 * p + 1));
      }
    }
  }
  s += __shfl_xor_sync(kFull, s, 1);
  s += __shfl_xor_sync(kFull, s, 2);
  if (x < k && p == 0 && HT_IN_RANGE(P, kChkString, 0, P.scr.cap_strings))
    atomicAdd(P.scr.str_acc + x, (unsigned long long)s);
}

}  // namespace ht
