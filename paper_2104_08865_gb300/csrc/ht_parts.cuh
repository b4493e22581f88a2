// ht_parts.cuh -- one string hashed in parts (on several devices or launches).
//
// A string of n bytes is cut at whole 64-execution chunks.  Each part runs the
// warp-chunk kernel over its chunks into a "part state": the context's tree
// scratch laid out as one array of 64-bit words (pending-root sums, packed
// 32-bit arrival counters, node accumulators).  Every entry is a sum over
// contributions, so the states of all parts add up element-wise (mod 2^64;
// the counters never exceed 8, so packed pairs do not carry) to the state of
// the whole string, except that groups whose children were split between parts
// have not been climbed yet.  The finish kernel climbs those, level by level
// (Section 5.2), and writes the digest.  The part holding the end of the
// string also adds the tail NH (Section 6.1), so finishing needs no input.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

// Adds the Toeplitz tail NH of the string in P.single (its tail bytes must be
// readable through P.single.ptr) to the pending-root sum.  One warp.
template <int W>
__global__ void __launch_bounds__(32) part_tail_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  constexpr uint64_t B = Dims<W>::exec_bytes;
  const int ln = threadIdx.x & 31;
  const StrPlan &sp = P.single;
  const uint64_t tstart = sp.n_exec * B;
  const uint64_t tlen = sp.len - tstart;
  const uint32_t M = (uint32_t)((tlen + 7) / 8);
  uint64_t sum[k];
#pragma unroll
  for (int t = 0; t < k; ++t) sum[t] = 0;
  for (uint32_t m = ln; m <= M; m += 32) {
    uint64_t word;
    if (m == M) {
      word = sp.len;
    } else {
      const uint64_t rem = tlen - 8ull * m;
      word = tail_word(sp.ptr + tstart + 8ull * m, rem < 8 ? (uint32_t)rem : 8u);
    }
#pragma unroll
    for (int t = 0; t < k; ++t) sum[t] += nh64(word, __ldg(P.seeds + Dims<W>::off_R + t + m));
  }
#pragma unroll
  for (int t = 0; t < k; ++t) sum[t] = warp_sum(sum[t]);
  if (ln == 0)
#pragma unroll
    for (int t = 0; t < k; ++t) atomicAdd(P.scr.str_acc + t, (unsigned long long)sum[t]);
}

// Finishes a merged part state of the string in P.single whose chunks have
// height L: every group that the merge completed (count 8) is climbed, parent
// levels in increasing order, then the digest is the pending-root sum.  One
// warp; thread (x, p) handles tree x, lanes 2p and 2p+1.
template <int W, int L>
__global__ void __launch_bounds__(32) part_finish_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  const int ln = threadIdx.x & 31;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = P.single.n_exec;
  uint64_t goff = 0;  // first group slot of parent level lvl + 1
  for (int lvl = L; lvl < kLevels - 1; ++lvl) {
    const uint64_t C = N >> (3 * lvl);
    const uint64_t groups = C >> 3;  // complete groups of level-lvl nodes
    for (uint64_t g0 = 0; g0 < groups; g0 += 32) {
      const uint64_t mine = g0 + ln;
      const bool done = mine < groups && __ldcg(P.scr.grp_cnt + goff + mine) == kFan;
      unsigned ballot = __ballot_sync(kFull, done);
      while (ballot) {
        const int b = __ffs(ballot) - 1;
        ballot &= ballot - 1;
        const uint64_t g = g0 + b;
        const uint64_t slot = goff + g;
        unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * kLanes + 2 * p;
        uint64_t v0 = 0, v1 = 0;
        if (x < k) {
          v0 = __ldcg(acc);
          v1 = __ldcg(acc + 1);
          acc[0] = 0;
          acc[1] = 0;
        }
        if (ln == 0) P.scr.grp_cnt[slot] = 0;
        // node (lvl + 1, g): pending, or one child of its parent
        const int plvl = lvl + 1;
        const uint64_t Cp = N >> (3 * plvl);
        const uint64_t first_pending = Cp & ~7ull;
        if (g >= first_pending) {
          const uint64_t j = g - first_pending;
          if (x < k)
            atomicAdd(P.scr.str_acc + x, (unsigned long long)(nh64(v0, final_key<W>(P, x, plvl, j, 2 * p)) +
                                                              nh64(v1, final_key<W>(P, x, plvl, j, 2 * p + 1))));
        } else {
          const int pos = (int)(g & 7);
          const uint64_t pslot = goff + groups + (g >> 3);
          unsigned long long *pacc = P.scr.grp_acc + (pslot * k + (uint64_t)x) * kLanes + 2 * p;
          if (x < k) {
            uint64_t a0 = v0, a1 = v1;
            if (pos < 7) {
              const uint64_t key = tree_key<W>(P, x, plvl, pos);
              a0 = nh64(v0, key);
              a1 = nh64(v1, key);
            }
            atomicAdd(pacc, (unsigned long long)a0);
            atomicAdd(pacc + 1, (unsigned long long)a1);
          }
          if (ln == 0) atomicAdd(P.scr.grp_cnt + pslot, 1u);
        }
        __threadfence();
        __syncwarp();
      }
    }
    goff += groups;
  }
  __threadfence();
  __syncwarp();
  if (ln < k) P.digests[ln] = __ldcg(P.scr.str_acc + ln);
}

}  // namespace ht
