// ht_stream.cuh -- the TMA-fed stream kernel of the HalftimeHash hot path.
//
// Work unit: a "stage" of 8 consecutive EHC executions of one string (one
// level-1 tree node), plus one data-less "tail unit" per string whose only job
// is to be counted.  The units of a launch (one string, or every string of a
// batch) form one sequence that is split into contiguous, equal ranges, one
// per warp, balanced to within one unit, so no warp idles at the end.
//
// Each warp owns a private ring of R shared-memory slots.  Lane 0 keeps up to
// R-1 stages in flight with one cp.async.bulk each (global -> shared, the
// mbarrier of the slot counts the bytes); all 32 lanes wait on the slot's
// mbarrier (bounded wait), hash the stage from shared memory and release the
// slot with __syncwarp.  Thread (x, p) handles execution x of the stage, lanes
// 2p and 2p+1.  Per stage:
//   * EHC (Section 3.3, Section 5.1) on each thread's two lanes;
//   * level 1 (Section 3.2 node variant, f = 8) by shuffles across x;
//   * level 2 accumulated in registers over the consecutive stages of one
//     64-execution chunk that fall into this warp's range.
// When a run of a chunk's children ends, the warp either holds the complete
// level-2 node (all 8 children) or adds the NH terms of the children it has,
// with their count, to the node's accumulator in scratch (64-bit atomics);
// the contribution that brings the count to 8 owns the node and climbs on.
// Nodes that never complete (base-8 digits of N, Eq. stack-construction) go
// straight into the string's final-NH sum; the warp whose unit count
// completes a string adds the Toeplitz tail (Section 6.1) and writes the
// digest.  Strings that are not 16-byte aligned are read with direct loads.
#pragma once

#include "ht_kernel.cuh"

namespace ht {

constexpr unsigned kStatusTimeout = 2;
// a wait on a stage's mbarrier gives up after ~1 s at 2 GHz
constexpr long long kWaitCycles = 2000000000ll;

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// One arrival without data (the checked build's stand-in for a skipped
// copy: the stage's phase still completes).
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Waits for the phase of `parity` to complete; false after `budget` cycles.
// The clock is read before every try (a try may itself suspend the thread
// for a while), so a budget of a few cycles runs out before the first try.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget = kWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 > budget) return false;
    uint32_t done;
    asm volatile(
        "{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

// EHC of one execution for lanes 2p, 2p+1 with the 21 (d*w) vectors supplied
// by `ld(blk)`.
template <int W, class Ld>
__device__ __forceinline__ void ehc2_from(Ld ld, const KParams &P, uint64_t (&y)[2][Spec<W>::k]) {
  using S = Spec<W>;
  constexpr int d = S::d, e = S::e, k = S::k, np = e - d, dw = d * kItemWords;
  uint4 v[dw];
#pragma unroll
  for (int b = 0; b < dw; ++b) v[b] = ld(b);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    uint32_t lo[dw], hi[dw];
#pragma unroll
    for (int b = 0; b < dw; ++b) {
      lo[b] = l ? v[b].z : v[b].x;
      hi[b] = l ? v[b].w : v[b].y;
    }
    uint64_t h[e];
#pragma unroll
    for (int c = 0; c < d; ++c) {
      h[c] = nh(lo[3 * c], hi[3 * c], P.E[3 * c]);
      h[c] += nh(lo[3 * c + 1], hi[3 * c + 1], P.E[3 * c + 1]);
      h[c] += nh(lo[3 * c + 2], hi[3 * c + 2], P.E[3 * c + 2]);
    }
#pragma unroll
    for (int r = 0; r < np; ++r) {
      h[d + r] = 0;
#pragma unroll
      for (int pv = 0; pv < 3; ++pv) {
        uint32_t plo = 0, phi = 0;
#pragma unroll
        for (int i = 0; i < d; ++i)
#pragma unroll
          for (int u = 0; u < 3; ++u)
            if (gf8_feeds(S::A(i, r), u, pv)) {
              plo ^= lo[3 * i + u];
              phi ^= hi[3 * i + u];
            }
        h[d + r] += nh(plo, phi, P.E[3 * (d + r) + pv]);
      }
    }
#pragma unroll
    for (int t = 0; t < k; ++t) y[l][t] = combine<W>(t, h);
  }
}

// Position of a warp in the unit sequence: string s, unit g of that string.
struct UnitCursor {
  unsigned s;
  uint64_t g;       // 0 .. stages-1: data units; == stages: the tail unit
  uint64_t stages;  // ceil(N / 8)
  StrPlan sp;
};

template <bool BATCH>
__device__ __forceinline__ void cursor_load(UnitCursor &c, const KParams &P, unsigned s) {
  c.s = s;
  c.sp = BATCH ? P.plans[s] : P.single;
  c.stages = (c.sp.n_exec + 7) >> 3;
}

template <bool BATCH>
__device__ __forceinline__ void cursor_seek(UnitCursor &c, const KParams &P, uint64_t u) {
  const unsigned s = BATCH ? find_string(P.item0s, P.count, u) : 0u;
  cursor_load<BATCH>(c, P, s);
  c.g = u - c.sp.item0;
}

template <bool BATCH>
__device__ __forceinline__ void cursor_next(UnitCursor &c, const KParams &P, bool more) {
  if (c.g == c.stages) {
    if (more) cursor_load<BATCH>(c, P, c.s + 1);
    c.g = 0;
  } else {
    ++c.g;
  }
}

__device__ __forceinline__ bool aligned16(const void *p) { return (((uintptr_t)p) & 15u) == 0; }

// Group accumulators for levels >= 2 are laid out level by level: the groups
// of level lvl+1 (parents of level-lvl nodes) follow those of lower levels.
__device__ __forceinline__ uint64_t group_offset(uint64_t N, int parent_lvl) {
  uint64_t off = 0;
  for (int l = 1; l < parent_lvl - 1; ++l) off += N >> (3 * l + 3);
  return off;
}

// Adds a final-NH term of tree t to string s's pending-root sum.  Pending
// roots are rare (at most 7 per level per string), so they go straight to
// the string's accumulator.
template <int W>
__device__ __forceinline__ void add_pending(const KParams &P, unsigned s, int t, uint64_t v) {
  atomicAdd(P.scr.str_acc + (uint64_t)s * Spec<W>::k + t, (unsigned long long)v);
}

// Node (lvl, idx) of string s (plan sp) is complete with value (v0, v1) for
// tree x, lanes 2p, 2p+1 (threads x >= k hold nothing).  Either it is
// pending (its final-NH term goes to the string's sum) or it is child
// idx & 7 of a parent: add its term, climb while we complete parents.
template <int W>
__device__ __noinline__ void push_node(const KParams &P, const StrPlan &sp, unsigned s, int lvl, uint64_t idx,
                          uint64_t v0, uint64_t v1, int ln) {
  constexpr int k = Spec<W>::k;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N = sp.n_exec;
  for (;;) {
    const uint64_t C = N >> (3 * lvl);
    const uint64_t first_pending = C & ~7ull;
    if (idx >= first_pending) {
      const uint64_t j = idx - first_pending;
      if (x < k)
        add_pending<W>(P, s, x, nh64(v0, final_key<W>(P, x, lvl, j, 2 * p)) +
                                    nh64(v1, final_key<W>(P, x, lvl, j, 2 * p + 1)));
      return;
    }
    const int pos = (int)(idx & 7);
    if (x < k && pos < 7) {
      const uint64_t key = tree_key<W>(P, x, lvl, pos);
      v0 = nh64(v0, key);
      v1 = nh64(v1, key);
    }
    // contribute one child to parent (lvl + 1, idx >> 3)
    const uint64_t slot = sp.grp0 + group_offset(N, lvl + 1) + (idx >> 3);
    unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * kLanes + 2 * p;
    if (x < k) {
      atomicAdd(acc, (unsigned long long)v0);
      atomicAdd(acc + 1, (unsigned long long)v1);
    }
    __threadfence();
    __syncwarp();
    unsigned old = 0;
    if (ln == 0) old = atomicAdd(P.scr.grp_cnt + slot, 1u);
    old = __shfl_sync(kFull, old, 0);
    if (old != kFan - 1) return;
    __threadfence();
    if (x < k) {
      v0 = ld_cg(acc);
      v1 = ld_cg(acc + 1);
      acc[0] = 0;
      acc[1] = 0;
    }
    if (ln == 0) P.scr.grp_cnt[slot] = 0;
    lvl += 1;
    idx >>= 3;
  }
}

// A run of n (1..7) consecutive children of the level-2 node `chunk` ended in
// this warp: add their summed terms (v0, v1 for tree x) with count n.
template <int W>
__device__ __noinline__ void contribute_level2(const KParams &P, const StrPlan &sp, unsigned s, uint64_t chunk,
                                  uint64_t v0, uint64_t v1, unsigned n, int ln) {
  constexpr int k = Spec<W>::k;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t slot = sp.grp0 + chunk;  // level-2 groups come first
  unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * kLanes + 2 * p;
  if (x < k) {
    atomicAdd(acc, (unsigned long long)v0);
    atomicAdd(acc + 1, (unsigned long long)v1);
  }
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0) old = atomicAdd(P.scr.grp_cnt + slot, n);
  old = __shfl_sync(kFull, old, 0);
  if (old + n != kFan) return;
  __threadfence();
  if (x < k) {
    v0 = ld_cg(acc);
    v1 = ld_cg(acc + 1);
    acc[0] = 0;
    acc[1] = 0;
  }
  if (ln == 0) P.scr.grp_cnt[slot] = 0;
  push_node<W>(P, sp, s, 2, chunk, v0, v1, ln);
}

template <int W, bool BATCH>
__global__ void __launch_bounds__(256) stream_kernel(const __grid_constant__ KParams P) {
  constexpr int k = Spec<W>::k;
  constexpr uint32_t B = Dims<W>::exec_bytes;
  constexpr uint32_t SLOT = 8 * B;
  extern __shared__ __align__(128) uint8_t smem[];
  const int ln = threadIdx.x & 31;
  const int x = ln >> 2, p = ln & 3;
  const unsigned R = P.stages;
  const unsigned wib = threadIdx.x >> 5;
  const uint32_t wbytes = ((R * (SLOT + 8)) + 127u) & ~127u;
  const uint32_t slots = (uint32_t)__cvta_generic_to_shared(smem) + wib * wbytes;
  const uint32_t bars = slots + R * SLOT;

  if (BATCH && __ldcg(&P.scr.ctl->status) != 0) return;
  // units of this launch: all units of the batch, or [item_begin, item_end)
  // of the single string
  const uint64_t ub = BATCH ? 0 : P.item_begin;
  const uint64_t U = BATCH ? __ldcg(&P.scr.ctl->total) : P.item_end - P.item_begin;
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const uint64_t nw = P.total_warps;
  const uint64_t q = U / nw, rr = U % nw;
  const uint64_t u_lo = ub + gw * q + (gw < rr ? gw : rr);
  const uint64_t u_hi = u_lo + q + (gw < rr ? 1 : 0);
  if (u_lo >= u_hi) return;

  if (ln == 0)
    for (unsigned i = 0; i < R; ++i) mbar_init(bars + 8 * i);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();

  // producer state (lane 0): next unit to consider and slot sequence numbers
  UnitCursor pc;
  uint64_t pu = u_lo, pseq = 0;
  if (ln == 0) cursor_seek<BATCH>(pc, P, u_lo);
  // consumer state
  UnitCursor cc;
  cursor_seek<BATCH>(cc, P, u_lo);
  uint64_t cseq = 0;
  bool failed = false;

  uint64_t pend[k];
#pragma unroll
  for (int t = 0; t < k; ++t) pend[t] = 0;
  bool anyp = false;
  uint64_t run[2][k];  // level-2 terms of the current run of children
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int t = 0; t < k; ++t) run[l][t] = 0;
  unsigned run_n = 0;
  uint64_t seg_units = 0;  // units of the current string done by this warp

  for (uint64_t u = u_lo; u < u_hi; ++u) {
    // keep R-1 stages in flight
    if (ln == 0 && !failed) {
      while (pu < u_hi && pseq < cseq + R) {
        const bool data = pc.g < pc.stages;
        if (data && aligned16(pc.sp.ptr)) {
          const uint64_t m = pc.sp.n_exec - 8 * pc.g < 8 ? pc.sp.n_exec - 8 * pc.g : 8;
          const unsigned sl = (unsigned)(pseq % R);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (HT_IN_RANGE(P, kChkInput, (8 * pc.g + m) * B - 1, pc.sp.len))
            bulk_load(slots + sl * SLOT, pc.sp.ptr + 8 * pc.g * B, (uint32_t)(m * B), bars + 8 * sl);
          else
            mbar_arrive(bars + 8 * sl);
          ++pseq;
        }
        ++pu;
        cursor_next<BATCH>(pc, P, pu < u_hi);
      }
    }
    const StrPlan &sp = cc.sp;
    const uint64_t N = sp.n_exec;
    const bool data = cc.g < cc.stages;
    if (data) {
      const uint64_t g = cc.g;
      const int m = (int)(N - 8 * g < 8 ? N - 8 * g : 8);
      uint64_t y[2][k];
      if (aligned16(sp.ptr)) {
        const unsigned sl = (unsigned)(cseq % R);
        if (!mbar_wait(bars + 8 * sl, (uint32_t)((cseq / R) & 1), P.wait_cycles > 0 ? P.wait_cycles : kWaitCycles))
          failed = true;
        failed = __any_sync(kFull, failed);
        if (failed) break;
        const uint32_t base = slots + sl * SLOT + x * B + p * 16;
        if (x < m) ehc2_from<W>([&](int b) { return lds128(base + b * 64); }, P, y);
        ++cseq;
      } else {
        const uint8_t *ex = sp.ptr + (8 * g + (uint64_t)x) * B + p * 16;
        const uint32_t sh = (uint32_t)(((uintptr_t)sp.ptr) & 15u);
        if (x < m && HT_IN_RANGE(P, kChkInput, (8 * g + (uint64_t)x + 1) * B - 1, sp.len))
          ehc2_from<W>([&](int b) { return ld_unaligned(ex + b * 64, sh); }, P, y);
      }
      if (m == 8) {
        uint64_t n1[2][k];
#pragma unroll
        for (int t = 0; t < k; ++t) {
          const uint64_t key = x < 7 ? tree_key<W>(P, t, 0, x) : 0;
#pragma unroll
          for (int l = 0; l < 2; ++l) n1[l][t] = x_sum(x < 7 ? nh64(y[l][t], key) : y[l][t]);
        }
        const uint64_t chunk = g >> 3;
        const int pos = (int)(g & 7);
        if (chunk < (N >> 6)) {
          // child pos of a level-2 node that will complete
#pragma unroll
          for (int t = 0; t < k; ++t) {
            const uint64_t key = pos < 7 ? tree_key<W>(P, t, 1, pos) : 0;
#pragma unroll
            for (int l = 0; l < 2; ++l) run[l][t] += pos < 7 ? nh64(n1[l][t], key) : n1[l][t];
          }
          ++run_n;
        } else {
          // level-1 node of the incomplete last chunk: pending, slot pos
#pragma unroll
          for (int t = 0; t < k; ++t)
            if (x == t)
              pend[t] += nh64(n1[0][t], final_key<W>(P, t, 1, pos, 2 * p)) +
                         nh64(n1[1][t], final_key<W>(P, t, 1, pos, 2 * p + 1));
          anyp = true;
        }
      } else if (x < m) {
        // leaves of the incomplete last stage: pending at level 0, slot x
#pragma unroll
        for (int t = 0; t < k; ++t)
          pend[t] += nh64(y[0][t], final_key<W>(P, t, 0, x, 2 * p)) +
                     nh64(y[1][t], final_key<W>(P, t, 0, x, 2 * p + 1));
        anyp = true;
      }
    }
    ++seg_units;
    const bool last_unit = (u + 1 == u_hi);
    const bool string_end = !data;  // the tail unit is a string's last unit
    // close the run of level-2 children at a chunk boundary or when this
    // warp leaves the chunk
    if (run_n > 0 && (((cc.g & 7) == 7) || last_unit || cc.g + 1 >= cc.stages)) {
      uint64_t v0 = 0, v1 = 0;
#pragma unroll
      for (int t = 0; t < k; ++t)
        if (x == t) {
          v0 = run[0][t];
          v1 = run[1][t];
        }
      const uint64_t chunk = cc.g >> 3;
      if (run_n == 8)
        push_node<W>(P, sp, cc.s, 2, chunk, v0, v1, ln);
      else
        contribute_level2<W>(P, sp, cc.s, chunk, v0, v1, run_n, ln);
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int t = 0; t < k; ++t) run[l][t] = 0;
      run_n = 0;
    }
    if (string_end || last_unit) {
      if (__any_sync(kFull, anyp)) {
#pragma unroll
        for (int t = 0; t < k; ++t) pend[t] = warp_sum(pend[t]);
        if (ln == 0)
#pragma unroll
          for (int t = 0; t < k; ++t)
            if (pend[t]) atomicAdd(P.scr.str_acc + (uint64_t)cc.s * k + t, (unsigned long long)pend[t]);
#pragma unroll
        for (int t = 0; t < k; ++t) pend[t] = 0;
        anyp = false;
      }
      __threadfence();
      __syncwarp();
      unsigned old = 0;
      if (ln == 0) old = atomicAdd(P.scr.str_done + cc.s, (unsigned)seg_units);
      old = __shfl_sync(kFull, old, 0);
      if ((uint64_t)old + seg_units == sp.n_items) finish_string<W>(P, sp, cc.s, ln);
      seg_units = 0;
    }
    __syncwarp();  // every lane is done with the slot before lane 0 refills it
    cursor_next<BATCH>(cc, P, !last_unit);
  }

  if (failed) {
    if (ln == 0) atomicOr(&P.scr.ctl->status, kStatusTimeout);
    // let the copies already issued land before the block's shared memory
    // is released (bounded as well, with the default limit)
    if (ln == 0)
      for (uint64_t sq = cseq; sq < pseq; ++sq) mbar_wait(bars + 8 * (unsigned)(sq % R), (uint32_t)((sq / R) & 1));
    __syncwarp();
  }
}

// A bounded wait that runs out, for testing the timeout path: one warp
// waits, with mbar_wait, on a shared-memory mbarrier that nothing arrives on
// and no copy completes, for `budget` cycles, then reports kStatusTimeout in
// the status word like the stream kernel does and returns.  (W only gives
// each width's table its own instance.)
template <int W>
__global__ void __launch_bounds__(32) wait_probe_kernel(Ctl *ctl, long long budget) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) mbar_init(b);
  __syncwarp();
  const bool ok = mbar_wait(b, 0, budget);
  if (!ok && threadIdx.x == 0) atomicOr(&ctl->status, kStatusTimeout);
}

}  // namespace ht
