// ht_block.cuh -- the block-chunk kernel: single strings of a few MiB to a few
// tens of MiB, where a launch is short and its fixed cost dominates.
//
// A block of eight warps takes one 64-execution chunk (the warp-chunk
// kernel's work item with L = 2): warp w hashes executions 8w .. 8w+7 of the
// chunk, one per x-thread (lanes 2p, 2p+1 in thread (x, p), as everywhere),
// and forms their level-1 node by shuffles across x; the chunk's level-2 node
// is formed from the eight warps' level-1 nodes in shared memory (Section
// 5.2 tree, f = 8, node variant of Section 3.2).  So a chunk costs one
// execution per thread instead of eight in a row, and the tree above it
// starts at level 2 (one level of cross-warp accumulation fewer than with
// 8-execution chunks).  Above the chunk the climb is the warp-chunk
// kernel's (atomic accumulators and arrival counts); the last warp to leave
// writes the digest.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

// INC: one update of an incremental handle (whole chunks only, the first
// possibly from the handle's buffer; pending nodes go to the stack, nothing
// is finished), as the warp-chunk kernel's incremental mode does it.  If the
// buffer holds only the first P.inc_fill bytes of that chunk (the rest
// start the update), block 0, whose first item it is, reads each of the
// chunk's executions from where its bytes are: the buffer, the update, or,
// for the one execution across the boundary, a copy in shared memory made
// by the block.  So no other kernel has to complete the chunk first.  The
// grid's last block only seeds the frontier groups from the previous
// stack, beside the chunk blocks instead of after one of them.
template <int W, bool ALIGNED, bool INC = false>
__global__ void __launch_bounds__(256, 2) block_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  constexpr uint64_t XB = Dims<W>::exec_bytes;
  __shared__ unsigned long long node1[8][k][kLanes];  // level-1 node of each warp
  __shared__ unsigned long long s_item;
  const int ln = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int x = ln >> 2, p = ln & 3;
  const StrPlan &sp = P.single;
  const uint64_t N = sp.n_exec;
  const uint32_t sh = ALIGNED ? 0u : (uint32_t)(((uintptr_t)sp.ptr) & 15u);
  // blocks that take chunks (an incremental update's last block seeds the
  // frontier instead)
  const unsigned nb = INC ? gridDim.x - 1 : gridDim.x;
  griddep_launch_dependents();
  bool first = true;
  for (;;) {
    uint64_t item;
    if (first) {
      if (INC && blockIdx.x == nb) break;
      item = P.item_begin + blockIdx.x;
      first = false;
    } else {
      if (P.item_end - P.item_begin <= nb) break;  // one round: nothing left to hand out
      __syncthreads();  // warp 0 is done with the previous chunk's nodes
      if (threadIdx.x == 0) s_item = atomicAdd(&P.scr.ctl->cursor, 1ull) + P.item_begin + nb;
      __syncthreads();
      item = s_item;
    }
    if (item >= P.item_end) break;
    uint64_t pend[k];  // this thread's share of the final-NH sum
#pragma unroll
    for (int t = 0; t < k; ++t) pend[t] = 0;
    bool anyp = false;
    const uint64_t e0 = item * 64;
    const uint64_t sb = e0 + 8ull * w;  // this warp's eight executions
    int m = sb >= N ? 0 : (int)((N - sb) < 8 ? (N - sb) : 8);
    const int M = e0 >= N ? 0 : (int)((N - e0) < 64 ? (N - e0) : 64);  // executions of the chunk
    const uint8_t *ex = sp.ptr + (sb + (uint64_t)x) * XB;  // this thread's execution
    uint32_t esh = sh;
    bool generic = false;  // ex is a generic (shared-memory) address
    if constexpr (INC) {
      if (P.inc_first && item == sp.chunk0) {
        // the update's first chunk: its first bytes were left in the handle's
        // buffer by the kernel before this one
        griddep_wait();
        const uint64_t e = 8ull * w + (uint64_t)x;  // the execution in the chunk
        if (!P.inc_fill) {
          ex = P.inc_first + e * XB;  // completed by a kernel before this one
          esh = 0;
        } else if constexpr (!ALIGNED) {
          __shared__ __align__(16) uint4 across[XB / 16];  // the execution across the boundary
          // (the buffer holds fewer bytes than a chunk; else nothing of the
          // chunk is read)
          const uint64_t fill = HT_IN_RANGE(P, kChkIncBuf, P.inc_fill, 64 * XB) ? P.inc_fill : 0;
          if (!fill) m = 0;
          const uint8_t *src = reinterpret_cast<const uint8_t *>(P.inc_stage_src);  // chunk byte fill
          const uint64_t ea = fill / XB;
          // (one granule per thread: XB / 16 <= 84 < 256)
          if (fill % XB && threadIdx.x < XB / 16)
            across[threadIdx.x] = chunk_granule(P.inc_first, src, fill, ea * XB + 16ull * threadIdx.x);
          __syncthreads();
          if ((e + 1) * XB <= fill) {
            ex = P.inc_first + e * XB;
            esh = 0;
          } else if (e * XB >= fill) {
            ex = src + (e * XB - fill);
            esh = (uint32_t)((uintptr_t)ex & 15u);
          } else {
            ex = reinterpret_cast<const uint8_t *>(across);
            esh = 0;
            generic = true;
          }
        }
      }
    }
    uint64_t y[2][k];
    if (x < m && HT_IN_RANGE(P, kChkInput, (sb + x + 1) * XB - 1, sp.len))
      ehc2<W, ALIGNED>(ex, p, esh, P, y, INC && generic);
    if (m == 8) {
      // level 1 across the eight x-threads; thread x = t keeps tree t: into
      // shared memory for level 2, or, in the string's last, incomplete
      // chunk, as a pending root of level 1, slot w
#pragma unroll
      for (int t = 0; t < k; ++t) {
        const uint64_t key = x < 7 ? tree_key<W>(P, t, 0, x) : 0;
        uint64_t n1[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) n1[l] = x_sum(x < 7 ? nh64(y[l][t], key) : y[l][t]);
        if (x == t) {
          if (M == 64) {
            node1[w][t][2 * p] = n1[0];
            node1[w][t][2 * p + 1] = n1[1];
          } else {
            pend[t] += nh64(n1[0], final_key<W>(P, t, 1, w, 2 * p)) +
                       nh64(n1[1], final_key<W>(P, t, 1, w, 2 * p + 1));
          }
        }
      }
      if (M < 64) anyp = true;
    } else if (x < m) {
      // the string's last, incomplete group of leaves: pending at level 0
#pragma unroll
      for (int t = 0; t < k; ++t)
        pend[t] += nh64(y[0][t], final_key<W>(P, t, 0, x, 2 * p)) +
                   nh64(y[1][t], final_key<W>(P, t, 0, x, 2 * p + 1));
      anyp = true;
    }
    __syncthreads();  // every warp's level-1 node is in shared memory
    // (scratch below: an overlapping launch first sees its predecessor end)
    griddep_wait();
    if (w == 0 && M == 64) {
      {
        // level 2 across the eight warps: thread (x, p), x < k, forms tree x,
        // lanes 2p and 2p+1, and climbs on
        uint64_t v0 = 0, v1 = 0;
        if (x < k) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint64_t a0 = node1[j][x][2 * p], a1 = node1[j][x][2 * p + 1];
            if (j < 7) {
              const uint64_t key = tree_key<W>(P, x, 1, j);
              v0 += nh64(a0, key);
              v1 += nh64(a1, key);
            } else {
              v0 += a0;
              v1 += a1;
            }
          }
        }
        climb<W, INC>(P, sp, 2, item, 0, v0, v1, ln, pend, anyp);
      }
    }
    flush_pending<W>(P, 0, pend, anyp, ln);
  }
  griddep_wait();
  if constexpr (INC) {
    // (its eight warps take the levels in turn: each level's arrivals and
    // climbs are independent of the others')
    if (blockIdx.x == nb) seed_frontier<W>(P, sp, ln, w, 8);
    // the bytes after the last whole chunk, for the next update
    if (HT_IN_RANGE(P, kChkIncBuf, P.inc_rem_len, 64 * XB))
      copy_bytes(P.inc_rem_dst, P.inc_rem_src, P.inc_rem_len, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
  }
  const bool last = exit_protocol(P, ln);
  if (!INC && last && P.item_end >= sp.n_items) finish_string<W>(P, sp, 0, ln);
}

}  // namespace ht
