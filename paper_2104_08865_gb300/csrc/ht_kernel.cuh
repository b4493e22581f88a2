// ht_kernel.cuh -- the HalftimeHash hot path for sm_103a (arXiv 2104.08865).
//
// One warp hashes one "chunk": 8^L consecutive EHC executions of one string
// (L = 1, 2 or 3).  Inside the chunk thread (x, p), x = lane>>2 in 0..7,
// p = lane&3 in 0..3, owns block lanes 2p and 2p+1 (one 16-byte load covers
// both) of execution x (L = 1) or of executions 8x..8x+7 of every
// 64-execution sub-chunk (L = 2, 3);
//   * EHC (Section 3.3, Section 5.1): 128-bit streaming loads, XOR-only
//     GF(8) encode, NH with mul.wide.u32 multiply-adds against keys held in
//     the constant bank, combine with the paper's small matrices;
//   * tree levels (Section 3.2 node variant, f = 8): with L = 1 level 1 by
//     warp shuffles across the eight x-threads; with L >= 2 level 1 in
//     registers, level 2 by shuffles, level 3 (L = 3) in registers again;
// Above the chunk, levels are finished across warps without waiting: every
// child adds its NH term of the parent (a sum, so order does not matter) into
// the parent's accumulator with 64-bit atomics and bumps the parent's arrival
// counter; the eighth arrival owns the parent and climbs on.  Nodes that can
// never complete (the base-8 digits of N, Eq. stack-construction) are folded
// straight into the string's final-NH sum (Section 5.2).  The warp that
// finishes a string's last work item adds the Toeplitz tail NH (Section 6.1)
// and writes the digest.  No kernel ever spins on another warp.
// With 256-bit blocks (template parameter B = 4, the block size of the
// paper's "v3" build, Section 6.3; L = 2 only) a work item is two
// 64-execution sub-chunks, one per half-warp, and thread (x, p) of a half is
// x = (lane >> 1) & 7, p = lane & 1.
#pragma once

#include "ht_check.cuh"
#include "ht_internal.h"
#include "ht_spec.cuh"

namespace ht {

constexpr unsigned kFull = 0xffffffffu;

// ---- arithmetic -------------------------------------------------------------

// NH of one 64-bit word (lo, hi) against one key word: (lo + s.lo)(hi + s.hi)
// with 32-bit sums and a 64-bit product (Section 3.2).
__device__ __forceinline__ uint64_t nh(uint32_t lo, uint32_t hi, uint64_t s) {
  return (uint64_t)(lo + (uint32_t)s) * (uint64_t)(hi + (uint32_t)(s >> 32));
}
__device__ __forceinline__ uint64_t nh64(uint64_t x, uint64_t s) {
  return nh((uint32_t)x, (uint32_t)(x >> 32), s);
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Thread roles in a warp for blocks of B words.  B = 8: thread (x, p),
// x = lane >> 2, p = lane & 3, owns block lanes 2p and 2p+1 of its
// executions.  B = 4 (256-bit blocks): the half-warps h = lane >> 4 take
// consecutive 64-execution sub-chunks, and in each thread (x, p),
// x = (lane >> 1) & 7, p = lane & 1, owns block lanes 2p and 2p+1.
template <int B>
__device__ __forceinline__ int lane_x(int ln) { return B == 8 ? ln >> 2 : (ln >> 1) & 7; }
template <int B>
__device__ __forceinline__ int lane_p(int ln) { return B == 8 ? ln & 3 : ln & 1; }
template <int B>
__device__ __forceinline__ int lane_h(int ln) { return B == 8 ? 0 : ln >> 4; }

// Sum over the eight x-threads that share (h, p): lane bits 2..4 for B = 8,
// lane bits 1..3 for B = 4.
template <int B = kLanes>
__device__ __forceinline__ uint64_t x_sum(uint64_t v) {
  constexpr int s = B == 8 ? 4 : 2;
  v += __shfl_xor_sync(kFull, v, s);
  v += __shfl_xor_sync(kFull, v, 2 * s);
  v += __shfl_xor_sync(kFull, v, 4 * s);
  return v;
}

__device__ __forceinline__ uint64_t ld_cg(const unsigned long long *p) {
  return __ldcg(p);
}

// Programmatic dependent launch: a launch that the host marked as allowed to
// overlap its predecessor in the stream waits here for that predecessor to
// finish (and its writes to be visible); without the mark this returns at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next launch in the stream start as soon as SM resources free up.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- loads ----------------------------------------------------------------------

// 16 bytes of input read once: no L1 allocation.
__device__ __forceinline__ uint4 ld_stream(const uint8_t *p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

// Bytes sh .. sh+15 (sh = 1..15) of the 32 bytes a, c (two consecutive
// aligned granules), by selects on the word offset and a funnel shift.
__device__ __forceinline__ uint4 realign(const uint4 a, const uint4 c, uint32_t sh) {
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
  uint32_t u[8], v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) u[j] = (sh & 8u) ? w[j + 2 < 8 ? j + 2 : 7] : w[j];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = (sh & 4u) ? u[j + 1 < 8 ? j + 1 : 7] : u[j];
  const uint32_t r = (sh & 3u) * 8u;
  uint4 o;
  o.x = __funnelshift_r(v[0], v[1], r);
  o.y = __funnelshift_r(v[1], v[2], r);
  o.z = __funnelshift_r(v[2], v[3], r);
  o.w = __funnelshift_r(v[3], v[4], r);
  return o;
}

// 16 bytes at an address that is not 16-byte aligned (sh = address & 15,
// 1..15): two aligned loads of the granules the bytes straddle, realigned.
// Both granules hold bytes of the request, so nothing outside the string's
// 16-byte granules is touched.
__device__ __forceinline__ uint4 ld_unaligned(const uint8_t *p, uint32_t sh) {
  const uint8_t *b = p - sh;
  return realign(ld_stream(b), ld_stream(b + 16), sh);
}

// Copies n bytes from src to dst (device memory, any alignments), shared by
// the caller's threads t = 0 .. nt-1: 16-byte stores over the part of dst
// that is 16-byte aligned (the source read with aligned loads and funnel
// shifts, touching only the 16-byte granules that hold source bytes), single
// bytes before and after it.
__device__ __forceinline__ void copy_bytes(uint8_t *dst, const uint8_t *src, uint64_t n, uint64_t t,
                                           uint64_t nt) {
  if (!n) return;
  const uintptr_t d0 = (uintptr_t)dst, d1 = d0 + n;
  const uintptr_t a0 = (d0 + 15) & ~(uintptr_t)15, a1 = d1 & ~(uintptr_t)15;
  if (a0 >= a1) {
    for (uint64_t i = t; i < n; i += nt) dst[i] = src[i];
    return;
  }
  const uint64_t head = a0 - d0, mid_end = a1 - d0;
  for (uint64_t i = t; i < head; i += nt) dst[i] = src[i];
  for (uint64_t i = mid_end + t; i < n; i += nt) dst[i] = src[i];
  const uint8_t *s = src + head;
  const uint32_t sh = (uint32_t)((uintptr_t)s & 15u);
  const uint64_t ng = (a1 - a0) >> 4;
  for (uint64_t g = t; g < ng; g += nt) {
    const uint4 v = sh ? ld_unaligned(s + 16 * g, sh) : ld_stream(s + 16 * g);
    *reinterpret_cast<uint4 *>(dst + head + 16 * g) = v;
  }
}

// 16 bytes at byte c (a multiple of 16) of an incremental update's first
// chunk, whose first `fill` bytes are in the handle's buffer and whose
// others start the update at src (any alignment): from either place, or,
// for the granule across the boundary, byte by byte.  (Not inlined: its
// registers stay out of the kernel's chunk loop.)
static __device__ __noinline__ uint4 chunk_granule(const uint8_t *buf, const uint8_t *src, uint64_t fill, uint64_t c) {
  if (c + 16 <= fill) return ld_stream(buf + c);
  if (c >= fill) {
    const uint8_t *q = src + (c - fill);
    const uint32_t qs = (uint32_t)((uintptr_t)q & 15u);
    return qs ? ld_unaligned(q, qs) : ld_stream(q);
  }
  uint32_t wd[4] = {0u, 0u, 0u, 0u};
  for (uint32_t b = 0; b < 16; ++b) {
    const uint64_t cb = c + b;
    const uint32_t byte = cb < fill ? __ldg(buf + cb) : __ldg(src + (cb - fill));
    wd[b >> 2] |= byte << (8 * (b & 3));
  }
  return make_uint4(wd[0], wd[1], wd[2], wd[3]);
}

// One little-endian word of the tail holding nb (1..8) bytes starting at p.
__device__ __forceinline__ uint64_t tail_word(const uint8_t *p, uint32_t nb) {
  if (nb == 8 && (((uintptr_t)p) & 7u) == 0)
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
  uint64_t w = 0;
  for (uint32_t i = 0; i < nb; ++i) w |= (uint64_t)__ldg(p + i) << (8 * i);
  return w;
}

// Row t of Combine, y_t = sum_c T[t][c] * h_c mod 2^64 (Section 5.1), as
// sum_c T*lo(h_c) + 2^32 * sum_c T*hi(h_c): a 64-bit multiply-add of the low
// halves (mad.wide.u32) and a 32-bit one of the high halves per nonzero
// coefficient, whatever the coefficient.
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

template <class S, int E>
__device__ __forceinline__ uint64_t combine_row_mad(int t, const uint64_t (&h)[E]) {
  uint64_t lo = 0;
  uint32_t hi = 0;
#pragma unroll
  for (int c = 0; c < E; ++c) {
    const uint32_t coef = (uint32_t)S::T(t, c);
    if (coef != 0) {
      lo = mad_wide(coef, (uint32_t)h[c], lo);
      hi += coef * (uint32_t)(h[c] >> 32);
    }
  }
  return lo + ((uint64_t)hi << 32);
}

// The same row as plain 64-bit arithmetic (the compiler picks shifts, adds
// and multiplies per coefficient).
template <class S, int E>
__device__ __forceinline__ uint64_t combine_row_plain(int t, const uint64_t (&h)[E]) {
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < E; ++c) {
    if (S::T(t, c) == 1) acc += h[c];
    else if (S::T(t, c) != 0) acc += (uint64_t)S::T(t, c) * h[c];
  }
  return acc;
}

// Measured on GB300: the split form is faster for width 32 (about 2%), the
// plain form for width 40; both are equal for widths 16 and 24.
template <int W, int E>
__device__ __forceinline__ uint64_t combine(int t, const uint64_t (&h)[E]) {
  if constexpr (W == 32) return combine_row_mad<Spec<W>>(t, h);
  else return combine_row_plain<Spec<W>>(t, h);
}

// ---- EHC ------------------------------------------------------------------------

// Realigns the dw granules v[b] of one unaligned execution (sh = 4Q +
// r8 / 8, 1..15): each thread's 16 bytes start sh bytes into its own granule
// and run into the next one, which the thread takes from its group
// neighbour src (that thread sends its own granule, or, if it is the
// group's first, the next block's granule, or `last` after the last block).
// Only the neighbour words the shift reaches (0 .. Q) are exchanged.
template <int Q, int dw>
__device__ __forceinline__ void realign_group(uint4 (&v)[dw], const uint4 last, int p, unsigned gmask,
                                              int src, uint32_t r8) {
#pragma unroll
  for (int b = 0; b < dw; ++b) {
    const uint4 out = p == 0 ? (b + 1 < dw ? v[b + 1] : last) : v[b];
    uint32_t n[4] = {0u, 0u, 0u, 0u};
    n[0] = __shfl_sync(gmask, out.x, src);
    if (Q >= 1) n[1] = __shfl_sync(gmask, out.y, src);
    if (Q >= 2) n[2] = __shfl_sync(gmask, out.z, src);
    if (Q >= 3) n[3] = __shfl_sync(gmask, out.w, src);
    const uint32_t w[8] = {v[b].x, v[b].y, v[b].z, v[b].w, n[0], n[1], n[2], n[3]};
    v[b].x = __funnelshift_r(w[Q], w[Q + 1], r8);
    v[b].y = __funnelshift_r(w[Q + 1], w[Q + 2], r8);
    v[b].z = __funnelshift_r(w[Q + 2], w[Q + 3], r8);
    v[b].w = __funnelshift_r(w[Q + 3], w[Q + 4], r8);
  }
}

// One EHC execution for block lanes 2p and 2p+1 (Section 3.3, Section 5.1):
// Encode (systematic GF(8) code, XOR only), Hash (NH of every encoded word
// under its own key E[c*3+u]), Combine (y = T h over Z_{2^64}).  Blocks are
// B words (8 B bytes) long.
template <int W, bool ALIGNED, int B = kLanes>
__device__ __forceinline__ void ehc2(const uint8_t *ex, int p, uint32_t sh,
                                     const KParams &P, uint64_t (&y)[2][Spec<W>::k], bool generic = false) {
  using S = Spec<W>;
  constexpr int d = S::d, e = S::e, k = S::k, np = e - d, dw = d * kItemWords;
  uint4 v[dw];
  if (ALIGNED || sh == 0) {
    // (generic: ex is a generic address, e.g. of shared memory, read with
    // plain loads)
#pragma unroll
    for (int b = 0; b < dw; ++b)
      v[b] = generic ? *reinterpret_cast<const uint4 *>(ex + b * (8 * B) + p * 16)
                     : ld_stream(ex + b * (8 * B) + p * 16);
  } else {
    // an unaligned execution: every aligned granule it touches is loaded
    // once, by the thread whose 16 bytes start in it; the granule after a
    // thread's own is its group neighbour's (p + 1), or, for the group's
    // last thread, the first one of the next block, loaded by thread 0 of
    // the group (one more granule past the last block: it still holds the
    // execution's last sh bytes).  All loads are in flight at once, as in
    // the aligned case, and the group exchanges granules by shuffles (the
    // group's threads always run ehc2 together).
    constexpr int G = B / 2;  // threads per block
    const int ln = (int)(threadIdx.x & 31);
    const int g0 = ln & ~(G - 1);
    const unsigned gmask = ((1u << G) - 1u) << g0;
    const int src = g0 + ((p + 1) & (G - 1));
    const uint8_t *a = ex - sh + p * 16;
#pragma unroll
    for (int b = 0; b < dw; ++b) v[b] = ld_stream(a + b * (8 * B));
    const uint4 last = p == 0 ? ld_stream(a + dw * (8 * B)) : make_uint4(0u, 0u, 0u, 0u);
    // (the word offset sh / 4 as a constant: only the neighbour's words
    // that the shift reaches are exchanged)
    const uint32_t r8 = (sh & 3u) * 8u;
    switch (sh >> 2) {
      case 0: realign_group<0>(v, last, p, gmask, src, r8); break;
      case 1: realign_group<1>(v, last, p, gmask, src, r8); break;
      case 2: realign_group<2>(v, last, p, gmask, src, r8); break;
      default: realign_group<3>(v, last, p, gmask, src, r8); break;
    }
  }
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

// ---- seeds ----------------------------------------------------------------------

template <int W>
__device__ __forceinline__ uint64_t tree_key(const KParams &P, int t, int lvl, int i) {
  const int r = (t * kLevels + lvl) * (kFan - 1) + i;
  if (!HT_IN_RANGE(P, kChkSeedT, r, Spec<W>::k * kLevels * (kFan - 1))) return 0;
  return __ldg(P.seeds + Dims<W>::off_T + r);
}
template <int W, int B = kLanes>
__device__ __forceinline__ uint64_t final_key(const KParams &P, int t, int lvl, uint64_t j, int lane) {
  const uint64_t r = ((uint64_t)(t * kLevels + lvl) * kFan + j) * B + lane;
  if (!HT_IN_RANGE(P, kChkSeedF, r, Spec<W>::k * kLevels * kFan * B)) return 0;
  return __ldg(P.seeds + Dims<W, B>::off_F + r);
}

// ---- the finaliser: pending-root sum + Toeplitz tail (Section 6.1) ----------

// The Toeplitz tail NH of the string, length word included (Section 6.1, and
// reading 9), summed over the warp: every lane gets the k sums.  BIN: the
// tail keys sit where the binary-tree ablation's seed layout puts them.
template <int W, int B = kLanes, bool BIN = false>
__device__ __forceinline__ void tail_sum(const KParams &P, const StrPlan &sp, int ln,
                                         uint64_t (&sum)[Spec<W>::k]) {
  constexpr int k = Spec<W>::k;
  constexpr int XB = Dims<W, B>::exec_bytes;
  constexpr int ROFF = BIN ? BinDims<W>::off_R : Dims<W, B>::off_R;
  const uint64_t tstart = sp.n_exec * (uint64_t)XB;
  const uint64_t tlen = sp.len - tstart;  // < B
  const uint32_t M = (uint32_t)((tlen + 7) / 8);
#pragma unroll
  for (int t = 0; t < k; ++t) sum[t] = 0;
  for (uint32_t m = ln; m <= M; m += 32) {
    uint64_t word = 0;
    if (m == M) {
      word = sp.len;
    } else {
      const uint64_t rem = tlen - 8ull * m;
      const uint32_t nb = rem < 8 ? (uint32_t)rem : 8u;
      if (HT_IN_RANGE(P, kChkInput, tstart + 8ull * m + nb - 1, sp.len))
        word = tail_word(sp.ptr + tstart + 8ull * m, nb);
    }
#pragma unroll
    for (int t = 0; t < k; ++t)
      if (HT_IN_RANGE(P, kChkSeedR, t + m, (B * Dims<W, B>::dw + k)))
        sum[t] += nh64(word, __ldg(P.seeds + ROFF + t + m));
  }
#pragma unroll
  for (int t = 0; t < k; ++t) sum[t] = warp_sum(sum[t]);
}

template <int W, int B = kLanes, bool BIN = false>
__device__ void finish_string(const KParams &P, const StrPlan &sp, unsigned sidx, int ln) {
  constexpr int k = Spec<W>::k;
  __threadfence();
  const bool str_ok = HT_IN_RANGE(P, kChkString, sidx, P.scr.cap_strings);
  uint64_t acc[k];
#pragma unroll
  for (int t = 0; t < k; ++t) acc[t] = str_ok ? ld_cg(P.scr.str_acc + (uint64_t)sidx * k + t) : 0;
  uint64_t sum[k];
  tail_sum<W, B, BIN>(P, sp, ln, sum);
  if (ln == 0 && str_ok) {
    const bool dig_ok = HT_IN_RANGE(P, kChkDigest, sidx, P.count);
#pragma unroll
    for (int t = 0; t < k; ++t) {
      if (dig_ok) P.digests[(uint64_t)sidx * k + t] = acc[t] + sum[t];
      P.scr.str_acc[(uint64_t)sidx * k + t] = 0;
    }
    P.scr.str_done[sidx] = 0;
  }
}

// A string with a single work item: its warp holds the whole final-NH sum
// (pend, spread over the lanes), so it writes the digest without the
// string's scratch sum and completion count.
template <int W, int B = kLanes, bool BIN = false>
__device__ void finish_local(const KParams &P, const StrPlan &sp, unsigned sidx,
                             uint64_t (&pend)[Spec<W>::k], int ln) {
  constexpr int k = Spec<W>::k;
  uint64_t sum[k];
  tail_sum<W, B, BIN>(P, sp, ln, sum);
#pragma unroll
  for (int t = 0; t < k; ++t) sum[t] += warp_sum(pend[t]);
  if (ln == 0 && HT_IN_RANGE(P, kChkDigest, sidx, P.count))
#pragma unroll
    for (int t = 0; t < k; ++t) P.digests[(uint64_t)sidx * k + t] = sum[t];
}

// ---- one work item: a chunk of 8^L executions ---------------------------------

constexpr uint64_t kNoNode = ~0ull;

// Levels 0..L of chunk c of a string (Section 5.2 tree, Eq. stack-construction)
// whose bytes start at base: the EHC values of its executions, level 1 in registers, level 2 across the
// eight x-threads, level 3 over eight sub-chunks (L = 3).  A full chunk's root
// (node c of level L) is returned in (v0, v1) of thread x < k (tree x, lanes
// 2p and 2p+1); the leaves and nodes of the string's last, incomplete chunk
// are pending roots, whose final NH goes into pend.  Returns whether the
// chunk is full.  Touches no scratch.
// With 256-bit blocks (B = 4, L = 2) a work item is two 64-execution
// sub-chunks, one per half-warp: half h returns level-2 node 2c + h.
template <int W, int L, bool ALIGNED, int B = kLanes>
__device__ __forceinline__ bool chunk_root(const KParams &P, const StrPlan &sp, const uint8_t *base,
                                           uint64_t c, int ln, uint64_t (&pend)[Spec<W>::k], bool &anyp,
                                           uint64_t &v0, uint64_t &v1) {
  static_assert(B == 8 || L == 2, "256-bit blocks take 64-execution sub-chunks");
  constexpr int k = Spec<W>::k;
  constexpr uint64_t XB = Dims<W, B>::exec_bytes;
  constexpr uint64_t CH = (uint64_t)(8 / B) << (3 * L);  // executions per work item
  const int x = lane_x<B>(ln), p = lane_p<B>(ln), h = lane_h<B>(ln);
  const uint64_t N = sp.n_exec;
  const uint32_t sh = ALIGNED ? 0u : (uint32_t)(((uintptr_t)base) & 15u);
  const bool full = c * CH < N && (N - c * CH) >= CH;
  const uint64_t e0 = c * CH;
  if (e0 >= N) return false;
  {
    uint64_t root[2][k];
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
      for (int t = 0; t < k; ++t) root[l][t] = 0;
    if constexpr (L == 1) {
      // eight executions, one per x-thread; level 1 across the x-threads
      const int m = (int)((N - e0) < 8 ? (N - e0) : 8);
      uint64_t y[2][k];
      if (x < m && HT_IN_RANGE(P, kChkInput, (e0 + x + 1) * XB - 1, sp.len))
        ehc2<W, ALIGNED>(base + (e0 + (uint64_t)x) * XB, p, sh, P, y);
      if (full) {
#pragma unroll
        for (int t = 0; t < k; ++t) {
          const uint64_t key = x < 7 ? tree_key<W>(P, t, 0, x) : 0;
#pragma unroll
          for (int l = 0; l < 2; ++l) root[l][t] = x_sum(x < 7 ? nh64(y[l][t], key) : y[l][t]);
        }
      } else if (x < m) {
        // the last, incomplete group of leaves: pending at level 0, slot x
#pragma unroll
        for (int t = 0; t < k; ++t)
          pend[t] += nh64(y[0][t], final_key<W>(P, t, 0, x, 2 * p)) +
                     nh64(y[1][t], final_key<W>(P, t, 0, x, 2 * p + 1));
        anyp = true;
      }
    }
    constexpr int NSUB = (L == 3) ? 8 : (L == 2 ? 1 : 0);
#pragma unroll 1
    for (int sub = 0; sub < NSUB; ++sub) {
      const uint64_t sb = e0 + 64ull * (sub + h);
      // (with B = 4 both half-warps stay for the shuffles below)
      if (B == 8 && sb >= N) break;
      const int m = sb >= N ? 0 : (int)((N - sb) < 64 ? (N - sb) : 64);
      int cnt = m - 8 * x;
      cnt = cnt < 0 ? 0 : (cnt > 8 ? 8 : cnt);
      uint64_t n1[2][k];
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int t = 0; t < k; ++t) n1[l][t] = 0;
      const uint8_t *ex = base + (sb + 8ull * x) * XB;
      if (cnt == 8) {
        // eight leaves -> one level-1 node per (tree, lane), in registers;
        // two executions per iteration keep two loads batches in flight
#pragma unroll (ALIGNED ? 2 : 1)
        for (int s = 0; s < 8; ++s) {
          uint64_t y[2][k];
          if (kChecked && !HT_IN_RANGE(P, kChkInput, (sb + 8ull * x + s + 1) * XB - 1, sp.len)) continue;
          ehc2<W, ALIGNED, B>(ex + s * XB, p, sh, P, y);
#pragma unroll
          for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int t = 0; t < k; ++t)
              n1[l][t] += (s < 7) ? nh64(y[l][t], P.T0[t][s]) : y[l][t];
        }
      } else {
        // the last, incomplete group of leaves: pending at level 0, slot s
#pragma unroll 1
        for (int s = 0; s < cnt; ++s) {
          uint64_t y[2][k];
          if (kChecked && !HT_IN_RANGE(P, kChkInput, (sb + 8ull * x + s + 1) * XB - 1, sp.len)) continue;
          ehc2<W, ALIGNED, B>(ex + s * XB, p, sh, P, y);
#pragma unroll
          for (int t = 0; t < k; ++t)
            pend[t] += nh64(y[0][t], final_key<W, B>(P, t, 0, s, 2 * p)) +
                       nh64(y[1][t], final_key<W, B>(P, t, 0, s, 2 * p + 1));
          anyp = true;
        }
      }
      if constexpr (B == 4) {
        // two sub-chunks, one per half-warp: the shuffles of level 2 run in
        // both halves whenever either half completes its level-2 node
        if (__any_sync(kFull, m == 64)) {
          uint64_t n2[2][k];
#pragma unroll
          for (int t = 0; t < k; ++t) {
            const uint64_t key = x < 7 ? tree_key<W>(P, t, 1, x) : 0;
#pragma unroll
            for (int l = 0; l < 2; ++l)
              n2[l][t] = x_sum<B>(x < 7 ? nh64(n1[l][t], key) : n1[l][t]);
          }
          if (m == 64 && full) {
#pragma unroll
            for (int l = 0; l < 2; ++l)
#pragma unroll
              for (int t = 0; t < k; ++t) root[l][t] = n2[l][t];
          } else if (m == 64) {
            // a complete level-2 node of an incomplete item: it lies in the
            // last, incomplete group of level 2, so it is pending there
            const uint64_t j = (2 * c + (uint64_t)h) - ((N >> 6) & ~7ull);
#pragma unroll
            for (int t = 0; t < k; ++t)
              if (x == t)
                pend[t] += nh64(n2[0][t], final_key<W, B>(P, t, 2, j, 2 * p)) +
                           nh64(n2[1][t], final_key<W, B>(P, t, 2, j, 2 * p + 1));
            anyp = true;
          }
        }
        if (m < 64 && cnt == 8) {
          // complete level-1 node of an incomplete sub-chunk: pending, slot x
#pragma unroll
          for (int t = 0; t < k; ++t)
            pend[t] += nh64(n1[0][t], final_key<W, B>(P, t, 1, x, 2 * p)) +
                       nh64(n1[1][t], final_key<W, B>(P, t, 1, x, 2 * p + 1));
          anyp = true;
        }
      } else if (m == 64) {
        // level 2 across the eight x-threads
        uint64_t n2[2][k];
#pragma unroll
        for (int t = 0; t < k; ++t) {
          const uint64_t key = x < 7 ? tree_key<W>(P, t, 1, x) : 0;
#pragma unroll
          for (int l = 0; l < 2; ++l)
            n2[l][t] = x_sum(x < 7 ? nh64(n1[l][t], key) : n1[l][t]);
        }
        if (L == 2) {
#pragma unroll
          for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int t = 0; t < k; ++t) root[l][t] = n2[l][t];
        } else if (full) {
#pragma unroll
          for (int t = 0; t < k; ++t) {
            const uint64_t key = sub < 7 ? tree_key<W>(P, t, 2, sub) : 0;
#pragma unroll
            for (int l = 0; l < 2; ++l)
              root[l][t] += sub < 7 ? nh64(n2[l][t], key) : n2[l][t];
          }
        } else {
          // a complete level-2 node of an incomplete chunk: pending, slot sub.
          // n2 is the same in all eight x-threads: thread x takes tree t = x.
#pragma unroll
          for (int t = 0; t < k; ++t)
            if (x == t)
              pend[t] += nh64(n2[0][t], final_key<W>(P, t, 2, sub, 2 * p)) +
                         nh64(n2[1][t], final_key<W>(P, t, 2, sub, 2 * p + 1));
          anyp = true;
        }
      } else if (cnt == 8) {
        // complete level-1 node of an incomplete sub-chunk: pending, slot x
#pragma unroll
        for (int t = 0; t < k; ++t)
          pend[t] += nh64(n1[0][t], final_key<W>(P, t, 1, x, 2 * p)) +
                     nh64(n1[1][t], final_key<W>(P, t, 1, x, 2 * p + 1));
        anyp = true;
      }
    }

    v0 = 0;
    v1 = 0;
#pragma unroll
    for (int t = 0; t < k; ++t)
      if (x == t) {
        v0 = root[0][t];
        v1 = root[1][t];
      }
  }
  return full;
}

// First group of level-lvl nodes that the launch's scratch holds (an
// incremental update counts from the group it starts in).
template <bool INC>
__device__ __forceinline__ uint64_t group_base(const StrPlan &sp, int lvl) {
  return INC ? (((sp.chunk0 << 6) >> (3 * lvl)) >> 3) : 0;
}

// Slot offset of level lvl + 1's groups, given level lvl's.
template <bool INC>
__device__ __forceinline__ uint64_t next_goff(const StrPlan &sp, int lvl, uint64_t goff) {
  return goff + ((sp.n_exec >> (3 * lvl)) >> 3) - group_base<INC>(sp, lvl);
}

// Node idx of level lvl, value (v0, v1) in thread x < k.  In the last,
// incomplete group of its level it is a pending root: its final NH goes into
// pend (or, in an incremental update, the node itself onto the stack, since
// its final position is not known yet).  Otherwise its contribution to its
// parent, NH under the tree key of its position (the eighth child enters
// unhashed), is added into the group's accumulator.
// Returns the group's slot, or kNoNode for a pending root.  With 256-bit
// blocks (B = 4) both half-warps hold the same node above the work item;
// the first half carries it.
template <int W, bool INC, int B = kLanes>
__device__ __forceinline__ uint64_t add_node(const KParams &P, const StrPlan &sp, int lvl, uint64_t idx,
                                             uint64_t goff, uint64_t v0, uint64_t v1, int ln,
                                             uint64_t (&pend)[Spec<W>::k], bool &anyp) {
  static_assert(!INC || B == 8, "incremental updates use 512-bit blocks");
  constexpr int k = Spec<W>::k;
  const int x = lane_x<B>(ln), p = lane_p<B>(ln);
  const bool own = lane_h<B>(ln) == 0;
  const uint64_t C = sp.n_exec >> (3 * lvl);
  const uint64_t first_pending = C & ~7ull;
  if (idx >= first_pending) {
    const uint64_t j = idx - first_pending;
    if constexpr (INC) {
      const uint64_t o = (((uint64_t)lvl * kFan + j) * k + (uint64_t)x) * kLanes + 2 * p;
      if (x < k && HT_IN_RANGE(P, kChkStack, o + 1, (uint64_t)kLevels * kFan * k * kLanes)) {
        P.stack[o] = v0;
        P.stack[o + 1] = v1;
      }
    } else {
#pragma unroll
      for (int t = 0; t < k; ++t)
        if (x == t && own)
          pend[t] += nh64(v0, final_key<W, B>(P, t, lvl, j, 2 * p)) +
                     nh64(v1, final_key<W, B>(P, t, lvl, j, 2 * p + 1));
      anyp = true;
    }
    return kNoNode;
  }
  const int pos = (int)(idx & 7);
  const uint64_t slot = sp.grp0 + goff + ((idx >> 3) - group_base<INC>(sp, lvl));
  if (x < k && own && HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups)) {
    unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * B + 2 * p;
    uint64_t a0 = v0, a1 = v1;
    if (pos < 7) {
      const uint64_t key = tree_key<W>(P, x, lvl, pos);
      a0 = nh64(v0, key);
      a1 = nh64(v1, key);
    }
    atomicAdd(acc, (unsigned long long)a0);
    atomicAdd(acc + 1, (unsigned long long)a1);
  }
  return slot;
}

// Counts n arrivals at a group (n children's contributions) after a fence
// that makes this warp's contributions visible; returns the count after
// them (all lanes).  The arrival that brings it to 8 completes the group.
__device__ __forceinline__ unsigned arrive(const KParams &P, uint64_t slot, int ln, unsigned n = 1) {
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0 && HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups)) old = atomicAdd(P.scr.grp_cnt + slot, n);
  return __shfl_sync(kFull, old, 0) + n;
}

// The warp that made the eighth arrival takes the group's node (its
// accumulator, then cleared for the next launch) into (v0, v1).
template <int W, int B = kLanes>
__device__ __forceinline__ void take_group(const KParams &P, uint64_t slot, int ln, uint64_t &v0, uint64_t &v1) {
  constexpr int k = Spec<W>::k;
  const int x = lane_x<B>(ln), p = lane_p<B>(ln);
  __threadfence();
  const bool ok = HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups);
  if (x < k && ok) {
    unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * B + 2 * p;
    v0 = ld_cg(acc);
    v1 = ld_cg(acc + 1);
    if (B == 8) {
      acc[0] = 0;
      acc[1] = 0;
    }
  }
  if (B == 4) {
    // both halves have read the node; the first clears it
    __syncwarp();
    if (x < k && lane_h<B>(ln) == 0 && ok) {
      unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * B + 2 * p;
      acc[0] = 0;
      acc[1] = 0;
    }
  }
  if (ln == 0 && ok) P.scr.grp_cnt[slot] = 0;
}

// Carries node idx of level lvl up the tree, waiting at every level: as long
// as this warp's arrival completes a group, it takes the parent node and goes
// on one level up.
template <int W, bool INC, int B = kLanes>
__device__ void climb(const KParams &P, const StrPlan &sp, int lvl, uint64_t idx, uint64_t goff,
                      uint64_t v0, uint64_t v1, int ln, uint64_t (&pend)[Spec<W>::k], bool &anyp) {
  for (;;) {
    const uint64_t slot = add_node<W, INC, B>(P, sp, lvl, idx, goff, v0, v1, ln, pend, anyp);
    if (slot == kNoNode) return;
    if (arrive(P, slot, ln) != kFan) return;
    take_group<W, B>(P, slot, ln, v0, v1);
    goff = next_goff<INC>(sp, lvl, goff);
    lvl += 1;
    idx >>= 3;
  }
}

// 256-bit blocks: the two level-2 nodes 2c and 2c+1 of a full work item c
// (one per half-warp) enter their common level-3 group as one arrival of two
// children -- each half adds the NH term of its own position, the first half
// adds the sum -- or, in the last, incomplete group, are pending roots.
// Returns the group's slot, or kNoNode.
template <int W>
__device__ __forceinline__ uint64_t add_pair(const KParams &P, const StrPlan &sp, uint64_t c,
                                             uint64_t v0, uint64_t v1, int ln,
                                             uint64_t (&pend)[Spec<W>::k], bool &anyp) {
  constexpr int k = Spec<W>::k, B = 4, lvl = 2;
  const int x = lane_x<B>(ln), p = lane_p<B>(ln), h = lane_h<B>(ln);
  const uint64_t idx0 = 2 * c, idx = idx0 + (uint64_t)h;
  const uint64_t first_pending = (sp.n_exec >> (3 * lvl)) & ~7ull;
  if (idx0 >= first_pending) {  // (idx0 and idx0 + 1 share a group)
    const uint64_t j = idx - first_pending;
#pragma unroll
    for (int t = 0; t < k; ++t)
      if (x == t)
        pend[t] += nh64(v0, final_key<W, B>(P, t, lvl, j, 2 * p)) +
                   nh64(v1, final_key<W, B>(P, t, lvl, j, 2 * p + 1));
    anyp = true;
    return kNoNode;
  }
  const int pos = (int)(idx & 7);
  const uint64_t slot = sp.grp0 + (idx0 >> 3);
  uint64_t a0 = v0, a1 = v1;
  if (x < k && pos < 7) {
    const uint64_t key = tree_key<W>(P, x, lvl, pos);
    a0 = nh64(v0, key);
    a1 = nh64(v1, key);
  }
  a0 += __shfl_xor_sync(kFull, a0, 16);
  a1 += __shfl_xor_sync(kFull, a1, 16);
  if (x < k && h == 0 && HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups)) {
    unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * B + 2 * p;
    atomicAdd(acc, (unsigned long long)a0);
    atomicAdd(acc + 1, (unsigned long long)a1);
  }
  return slot;
}

// The root(s) of full work item c enter the tree above the item and climb.
template <int W, int L, int B>
__device__ __forceinline__ void climb_item(const KParams &P, const StrPlan &sp, uint64_t c, uint64_t v0,
                                           uint64_t v1, int ln, uint64_t (&pend)[Spec<W>::k], bool &anyp) {
  if constexpr (B == 8) {
    climb<W, false>(P, sp, L, c, 0, v0, v1, ln, pend, anyp);
  } else {
    static_assert(L == 2, "256-bit blocks take 64-execution sub-chunks");
    const uint64_t slot = add_pair<W>(P, sp, c, v0, v1, ln, pend, anyp);
    if (slot == kNoNode) return;
    if (arrive(P, slot, ln, 2) != kFan) return;
    take_group<W, B>(P, slot, ln, v0, v1);
    climb<W, false, B>(P, sp, L + 1, (2 * c) >> 3, next_goff<false>(sp, L, 0), v0, v1, ln, pend, anyp);
  }
}

// Adds this warp's share of a string's final-NH sum into the string's sum.
template <int W>
__device__ __forceinline__ void flush_pending(const KParams &P, unsigned sidx, uint64_t (&pend)[Spec<W>::k],
                                              bool anyp, int ln) {
  constexpr int k = Spec<W>::k;
  if (__any_sync(kFull, anyp)) {
#pragma unroll
    for (int t = 0; t < k; ++t) pend[t] = warp_sum(pend[t]);
    if (ln == 0 && HT_IN_RANGE(P, kChkString, sidx, P.scr.cap_strings))
#pragma unroll
      for (int t = 0; t < k; ++t)
        if (pend[t]) atomicAdd(P.scr.str_acc + (uint64_t)sidx * k + t, (unsigned long long)pend[t]);
  }
}

// One chunk of a batch: its levels, the climb, and the string's completion
// count (the warp that completes the string runs the finaliser).
template <int W, int L, bool ALIGNED, int B = kLanes>
__device__ void hash_chunk(const KParams &P, const StrPlan &sp, unsigned sidx, uint64_t c, int ln) {
  constexpr int k = Spec<W>::k;
  uint64_t pend[k];  // this thread's share of the final-NH sum
#pragma unroll
  for (int t = 0; t < k; ++t) pend[t] = 0;
  bool anyp = false;
  uint64_t v0, v1;
  const bool full = chunk_root<W, L, ALIGNED, B>(P, sp, sp.ptr, c, ln, pend, anyp, v0, v1);
  griddep_wait();
  if (full) climb_item<W, L, B>(P, sp, c, v0, v1, ln, pend, anyp);
  if (sp.n_items == 1) {
    // (a single chunk's root is a pending root: the climb touched no scratch)
    finish_local<W, B>(P, sp, sidx, pend, ln);
    return;
  }
  flush_pending<W>(P, sidx, pend, anyp, ln);
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0 && HT_IN_RANGE(P, kChkString, sidx, P.scr.cap_strings)) old = atomicAdd(P.scr.str_done + sidx, 1u);
  old = __shfl_sync(kFull, old, 0);
  if (old == sp.n_items - 1) finish_string<W, B>(P, sp, sidx, ln);
}

// Incremental update, the frontier: the stack carries, for every level, the
// nodes of its last, incomplete group (d of them).  If the update completes
// that group, the d nodes enter it as one arrival of d children (the sum of
// their tree-key NH terms); arrivals are sums and counts, so the order
// against the chunks' own arrivals does not matter, and whichever brings the
// count to 8 takes the parent node and climbs on.  Otherwise the d nodes stay
// pending and are copied to the same positions of the new stack (the
// update's own pending nodes of that level come after them).  The previous
// stack is only read, so no other warp's writes can race with this.  The
// levels are independent of one another (a node climbing out of one level
// arrives in the next one's group beside its stack nodes, at a position the
// copy does not touch), so several warps may split them.
template <int W>
__device__ void seed_frontier(const KParams &P, const StrPlan &sp, int ln, int part = 0, int parts = 1) {
  constexpr int k = Spec<W>::k;
  const int x = ln >> 2, p = ln & 3;
  const uint64_t N0 = sp.chunk0 << 6, N1 = sp.n_exec;
  uint64_t goff = 0;
  for (int lvl = 2; lvl < kLevels; ++lvl) {
    // (levels are independent: warp `part` of `parts` takes every parts-th)
    if ((lvl - 2) % parts != part) {
      if (lvl < kLevels - 1) goff = next_goff<true>(sp, lvl, goff);
      continue;
    }
    const uint64_t n0 = N0 >> (3 * lvl), n1 = N1 >> (3 * lvl);
    const unsigned d = (unsigned)(n0 & 7);
    const bool completes = (n1 >> 3) > (n0 >> 3);
    if (d && !completes) {
      if (x < k)
        for (unsigned j = 0; j < d; ++j) {
          const uint64_t o = (((uint64_t)lvl * kFan + j) * k + (uint64_t)x) * kLanes + 2 * p;
          if (!HT_IN_RANGE(P, kChkStack, o + 1, (uint64_t)kLevels * kFan * k * kLanes)) continue;
          P.stack[o] = P.stack_in[o];
          P.stack[o + 1] = P.stack_in[o + 1];
        }
    } else if (d) {
      const uint64_t slot = sp.grp0 + goff;  // the level's first group slot
      if (x < k) {
        uint64_t a0 = 0, a1 = 0;
        for (unsigned j = 0; j < d; ++j) {  // j < 7: every stack node is hashed
          const uint64_t key = tree_key<W>(P, x, lvl, (int)j);
          const uint64_t o = (((uint64_t)lvl * kFan + j) * k + (uint64_t)x) * kLanes + 2 * p;
          if (!HT_IN_RANGE(P, kChkStack, o + 1, (uint64_t)kLevels * kFan * k * kLanes)) continue;
          a0 += nh64(P.stack_in[o], key);
          a1 += nh64(P.stack_in[o + 1], key);
        }
        if (HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups)) {
          unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * kLanes + 2 * p;
          atomicAdd(acc, (unsigned long long)a0);
          atomicAdd(acc + 1, (unsigned long long)a1);
        }
      }
      if (arrive(P, slot, ln, d) == kFan) {
        uint64_t pend[k];  // (unused: incremental pending nodes go to the stack)
        bool anyp = false;
        uint64_t v0 = 0, v1 = 0;
        take_group<W>(P, slot, ln, v0, v1);
        climb<W, true>(P, sp, lvl + 1, n0 >> 3, next_goff<true>(sp, lvl, goff), v0, v1, ln, pend, anyp);
      }
    }
    if (lvl < kLevels - 1) goff = next_goff<true>(sp, lvl, goff);
  }
}

// One of the eight warps that hash an incremental update's first chunk
// (complete: 64 executions) when the handle's buffer holds only its first
// `fill` bytes and the others start the update at src: warp j takes level-1
// node j, thread x execution 8j + x, read where its bytes are (the buffer,
// the update at any alignment, or, for the execution across the boundary, a
// copy the warp makes in shared memory), forms the node by shuffles and adds
// its NH term in the chunk's level-2 node to group slot `slot` (one arrival);
// the eighth arrival takes the level-2 node and climbs from there.  Eight
// warps side by side instead of one warp's eight executions in a row.
template <int W>
__device__ __forceinline__ void inc_chunk0_part(const KParams &P, const StrPlan &sp, int j, uint64_t slot,
                                                int ln) {
  constexpr int k = Spec<W>::k;
  constexpr uint64_t XB = Dims<W>::exec_bytes;
  __shared__ __align__(16) uint4 across[XB / 16];  // (one warp per block uses it)
  const int x = ln >> 2, p = ln & 3;
  const uint8_t *buf = P.inc_first;
  const uint64_t fill = P.inc_fill;
  const uint8_t *src = reinterpret_cast<const uint8_t *>(P.inc_stage_src);
  const uint64_t ea = fill / XB;  // the execution across the boundary (if fill % XB)
  if (fill % XB && (uint64_t)j == ea / 8)
    for (uint32_t g = (uint32_t)ln; g < XB / 16; g += 32) across[g] = chunk_granule(buf, src, fill, ea * XB + 16ull * g);
  __syncwarp();
  const uint64_t e = 8ull * j + x;
  const uint8_t *ex;
  uint32_t esh = 0;
  bool generic = false;
  if ((e + 1) * XB <= fill) {
    ex = buf + e * XB;
  } else if (e * XB >= fill) {
    ex = src + (e * XB - fill);
    esh = (uint32_t)((uintptr_t)ex & 15u);
  } else {
    ex = reinterpret_cast<const uint8_t *>(across);
    generic = true;
  }
  uint64_t y[2][k];
  ehc2<W, false>(ex, p, esh, P, y, generic);
  uint64_t a0 = 0, a1 = 0;
#pragma unroll
  for (int t = 0; t < k; ++t) {
    const uint64_t key = x < 7 ? tree_key<W>(P, t, 0, x) : 0;
    const uint64_t n0 = x_sum(x < 7 ? nh64(y[0][t], key) : y[0][t]);
    const uint64_t n1 = x_sum(x < 7 ? nh64(y[1][t], key) : y[1][t]);
    if (x == t) {
      // node j's term in the level-2 node (the eighth child enters unhashed)
      const uint64_t key2 = j < 7 ? tree_key<W>(P, t, 1, j) : 0;
      a0 = j < 7 ? nh64(n0, key2) : n0;
      a1 = j < 7 ? nh64(n1, key2) : n1;
    }
  }
  if (x < k && HT_IN_RANGE(P, kChkGroup, slot, P.scr.cap_groups)) {
    unsigned long long *acc = P.scr.grp_acc + (slot * k + (uint64_t)x) * kLanes + 2 * p;
    atomicAdd(acc, (unsigned long long)a0);
    atomicAdd(acc + 1, (unsigned long long)a1);
  }
  if (arrive(P, slot, ln, 1) == kFan) {
    uint64_t pend[k];  // (unused: incremental pending nodes go to the stack)
    bool anyp = false;
    uint64_t v0 = 0, v1 = 0;
    take_group<W>(P, slot, ln, v0, v1);
    climb<W, true>(P, sp, 2, sp.chunk0, 0, v0, v1, ln, pend, anyp);
  }
}

// A warp's share of one string (single-string launches, incremental updates):
// chunks from the cursor, each root climbing as far as this warp completes
// groups.  Completion of the string needs no count per chunk (a fence and an
// L2 round trip the warp would wait on): the last warp to leave the launch
// that ends the string runs the finaliser.  An incremental update may take
// its first chunk from the buffer of bytes carried over from earlier updates
// (P.inc_first), and its first warp seeds the frontier groups.
template <int W, int L, bool ALIGNED, bool INC, int B = kLanes>
__device__ __forceinline__ void single_string(const KParams &P, uint64_t gw, int ln) {
  static_assert(!INC || B == 8, "incremental updates use 512-bit blocks");
  constexpr int k = Spec<W>::k;
  constexpr uint64_t G = (1ull << (3 * L)) * Dims<W>::exec_bytes;
  const StrPlan &sp = P.single;
  // warps that take chunks: in an incremental update the last warp seeds the
  // frontier instead, beside them, and, when the buffer holds only part of
  // the update's first chunk, the eight warps before it hash that chunk
  // (the others start at the chunk after it)
  const uint64_t extra = INC ? (P.inc_fill ? 9 : 1) : 0;
  const uint64_t cw = P.total_warps - extra;
  bool first = true;
  for (;;) {
    unsigned long long item = 0;
    if (first) {
      // each warp's first chunk is fixed, so it can be hashed before an
      // overlapping launch's predecessor has finished with the scratch
      if (INC && gw >= cw) break;
      item = P.item_begin + gw;
      first = false;
    } else {
      // a launch of one round hands nothing out through the cursor
      if (P.item_end - P.item_begin <= cw) break;
      if (ln == 0) item = atomicAdd(&P.scr.ctl->cursor, 1ull);
      item = __shfl_sync(kFull, item, 0) + P.item_begin + cw;
    }
    if (item >= P.item_end) break;
    uint64_t pend[k];  // this thread's share of the final-NH sum
#pragma unroll
    for (int t = 0; t < k; ++t) pend[t] = 0;
    bool anyp = false;
    uint64_t v0, v1;
    const uint8_t *base = sp.ptr;
    if constexpr (INC) {
      if (P.inc_first && item == sp.chunk0) {
        // the update's first chunk, completed in the handle's buffer by the
        // kernel before this one
        griddep_wait();
        base = P.inc_first - item * G;
      }
    }
    const bool full = chunk_root<W, L, ALIGNED, B>(P, sp, base, item, ln, pend, anyp, v0, v1);
    // everything below touches the scratch: an overlapping launch must first
    // see its predecessor finish
    griddep_wait();
    if (full) {
      if constexpr (INC) climb<W, INC>(P, sp, L, item, 0, v0, v1, ln, pend, anyp);
      else climb_item<W, L, B>(P, sp, item, v0, v1, ln, pend, anyp);
    }
    flush_pending<W>(P, 0, pend, anyp, ln);
  }
  griddep_wait();
  if constexpr (INC) {
    if (gw == P.total_warps - 1) seed_frontier<W>(P, sp, ln);
    if constexpr (!ALIGNED) {
      // (the buffer holds fewer bytes than a chunk; else nothing of the
      // chunk is read)
      if (P.inc_fill && gw >= cw && gw < cw + 8 && HT_IN_RANGE(P, kChkIncBuf, P.inc_fill, G))
        inc_chunk0_part<W>(P, sp, (int)(gw - cw), P.inc_chunk0_slot, ln);
    }
    // the bytes after the last whole chunk, for the next update
    if (HT_IN_RANGE(P, kChkIncBuf, P.inc_rem_len, G))
      copy_bytes(P.inc_rem_dst, P.inc_rem_src, P.inc_rem_len, 32 * gw + ln, 32ull * P.total_warps);
  }
}

// ---- the persistent kernel ----------------------------------------------------

__device__ __forceinline__ unsigned find_string(const unsigned long long *item0s,
                                                unsigned count, uint64_t item) {
  unsigned lo = 0, hi = count;  // item0s[lo] <= item < item0s[hi]
  while (hi - lo > 1) {
    const unsigned mid = (lo + hi) >> 1;
    if (__ldg(item0s + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// The same search by a whole (converged) warp: every step probes 32 evenly
// spaced entries of (lo, hi] at once, lane j at lo + span (j + 1) / 32 (lane
// 31 at hi, known to be > item, and not loaded), and keeps the interval
// between the last probe <= item and the first one > item: about 32 times
// smaller, so 50,000 strings take 4 dependent loads instead of 16.
__device__ __forceinline__ unsigned find_string_warp(const unsigned long long *item0s,
                                                     unsigned count, uint64_t item, int ln) {
  unsigned lo = 0, hi = count;  // item0s[lo] <= item < item0s[hi]
  while (hi - lo > 1) {
    const uint64_t span = hi - lo;
    const unsigned pos = lo + (unsigned)((span * (unsigned)(ln + 1)) >> 5);
    const bool le = pos < hi && __ldg(item0s + pos) <= item;
    const unsigned j = (unsigned)__popc(__ballot_sync(kFull, le));  // probes 0 .. j-1 are <= item
    const unsigned nlo = lo + (unsigned)((span * j) >> 5);
    hi = lo + (unsigned)((span * (j + 1)) >> 5);
    lo = nlo;
  }
  return lo;
}

// Every warp passes here on leaving; the last one (all other warps' work is
// then visible to it) rearms the cursor for the next launch and learns that
// it was last.
__device__ __forceinline__ bool exit_protocol(const KParams &P, int ln) {
  griddep_wait();
  __syncwarp();
  unsigned old = 0;
  if (ln == 0) {
    __threadfence();
    old = atomicAdd(&P.scr.ctl->exit, 1u);
    if (old == P.total_warps - 1) {
      P.scr.ctl->cursor = 0;
      P.scr.ctl->exit = 0;
      __threadfence();
    }
  }
  return __shfl_sync(kFull, old, 0) == P.total_warps - 1;
}

// B: words per block, 8 (the default, 512-bit blocks) or 4 (256-bit blocks).
// MAP (batches): find each work item's string in the planner's item map
// (one load) instead of searching the prefix sums; a separate instance,
// used for batches of many strings, so that the searching one keeps its code.
template <int W, int L, bool SINGLE, bool ALIGNED, bool INC = false, int B = kLanes, bool MAP = false>
__global__ void __launch_bounds__(256, 2) hash_kernel(const __grid_constant__ KParams P) {
  static_assert(!INC || (SINGLE && L == 2), "incremental updates hash one string in 64-execution chunks");
  const int ln = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if constexpr (SINGLE) {
    griddep_launch_dependents();
    single_string<W, L, ALIGNED, INC, B>(P, gw, ln);
    const bool last = exit_protocol(P, ln);
    // nothing is final in an incremental update; a string hashed over several
    // launches ends with the launch that reaches its item count (parts of a
    // split string set an unreachable count: they are finished elsewhere)
    if (!INC && last && P.item_end >= P.single.n_items) finish_string<W, B>(P, P.single, 0, ln);
    return;
  } else {
    // a batch runs an aligned-only and a general variant; the planner's
    // alignment flag selects one, the other leaves at once
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
      unsigned s;
      if constexpr (MAP) s = __ldg(P.item_str + item);
      else s = find_string_warp(P.item0s, P.count, item, ln);
      const StrPlan sp = P.plans[s];
      const uint64_t c = item - sp.item0;
      if (ALIGNED || (((uintptr_t)sp.ptr) & 15u) == 0)
        hash_chunk<W, L, true, B>(P, sp, s, c, ln);
      else
        hash_chunk<W, L, false, B>(P, sp, s, c, ln);
    }
    exit_protocol(P, ln);
  }
}

// ---- the batch planner (one block) ---------------------------------------------

// Block-wide exclusive scan of one value per thread (1024 threads at most);
// returns the exclusive prefix and writes the total to *total.
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, unsigned long long *sh,
                                                         unsigned long long *total) {
  const unsigned tid = threadIdx.x, nt = blockDim.x;
  const int ln = tid & 31, wid = tid >> 5;
  unsigned long long xi = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFull, xi, o);
    if (ln >= o) xi += y;
  }
  __syncthreads();
  if (ln == 31) sh[wid] = xi;
  __syncthreads();
  if (wid == 0) {
    const unsigned nw = nt >> 5;
    unsigned long long w = ln < (int)nw ? sh[ln] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, w, o);
      if (ln >= o) w += y;
    }
    if (ln < (int)nw) sh[ln] = w;
  }
  __syncthreads();
  const unsigned long long excl = (xi - v) + (wid ? sh[wid - 1] : 0);
  *total = sh[(nt >> 5) - 1];
  __syncthreads();
  return excl;
}

// The batch planner (one block of 1024 threads): per string, executions N,
// work units (L = 0: stream/range units, one per 8 executions plus the tail
// unit; L >= 1: warp-chunk items of 8^L executions), tree-group slots, full
// 64-execution chunks, and their prefix sums; then the hybrid kernel's work
// list: phase A holds every full chunk of the batch but the last
// total_warps, phase B every remaining unit.
template <int W, int L>
__global__ void __launch_bounds__(1024) plan_kernel(const PlanArgs A) {
  constexpr uint64_t B = Dims<W>::exec_bytes;
  __shared__ unsigned long long sh[32];
  const unsigned tid = threadIdx.x, nt = blockDim.x;
  const unsigned per = (A.count + nt - 1) / nt;
  const unsigned lo = tid * per < A.count ? tid * per : A.count;
  const unsigned hi = lo + per < A.count ? lo + per : A.count;
  auto groups_of = [](uint64_t N) -> unsigned long long {
    uint64_t g = 0;
    for (int lvl = (L == 0 ? 1 : L); lvl < kLevels; ++lvl) g += N >> (3 * lvl + 3);
    return g;
  };
  auto items_of = [](uint64_t N) -> unsigned long long {
    if (L == 0) return ((N + 7) >> 3) + 1;
    const uint64_t it = (N + (1ull << (3 * L)) - 1) >> (3 * L);
    return it ? it : 1ull;
  };
  unsigned long long my_items = 0, my_groups = 0, my_chunks = 0;
  bool my_unaligned = false;
  for (unsigned i = lo; i < hi; ++i) {
    const uint64_t N = A.lens[i] / B;
    my_items += items_of(N);
    my_groups += groups_of(N);
    my_chunks += N >> 6;
    my_unaligned |= (((uintptr_t)A.ptrs[i]) & 15u) != 0;
  }
  const int any_unaligned = __syncthreads_or(my_unaligned);
  unsigned long long total_i, total_g, total_c;
  unsigned long long base_i = block_scan(my_items, sh, &total_i);
  unsigned long long base_g = block_scan(my_groups, sh, &total_g);
  unsigned long long base_c = block_scan(my_chunks, sh, &total_c);
  // phase A: every full chunk but the last nw (one per warp), whole
  const unsigned long long nw = A.total_warps ? A.total_warps : 1;
  const unsigned long long cut = total_c > nw ? total_c - nw : 0;
  unsigned long long my_b = 0;
  {
    unsigned long long c0 = base_c;
    for (unsigned i = lo; i < hi; ++i) {
      const uint64_t N = A.lens[i] / B;
      const unsigned long long C2 = N >> 6;
      const unsigned long long a = cut > c0 ? (cut - c0 < C2 ? cut - c0 : C2) : 0;
      my_b += items_of(N) - 8 * a;
      c0 += C2;
    }
  }
  unsigned long long total_b;
  unsigned long long base_b = block_scan(my_b, sh, &total_b);
  for (unsigned i = lo; i < hi; ++i) {
    const uint64_t len = A.lens[i];
    const uint64_t N = len / B;
    const unsigned long long C2 = N >> 6;
    const unsigned long long a = cut > base_c ? (cut - base_c < C2 ? cut - base_c : C2) : 0;
    StrPlan sp;
    sp.ptr = static_cast<const uint8_t *>(A.ptrs[i]);
    sp.len = len;
    sp.n_exec = N;
    sp.item0 = base_i;
    sp.grp0 = base_g;
    sp.n_items = (uint32_t)items_of(N);
    sp.pad = 0;
    sp.chunk0 = base_c;
    sp.chunks_a = a;
    sp.unitb0 = base_b;
    A.plans[i] = sp;
    A.item0s[i] = base_i;
    A.chunk0s[i] = base_c;
    A.unitb0s[i] = base_b;
    base_i += items_of(N);
    base_g += groups_of(N);
    base_c += C2;
    base_b += items_of(N) - 8 * a;
  }
  if (tid == nt - 1) {
    A.item0s[A.count] = total_i;
    A.chunk0s[A.count] = total_c;
    A.unitb0s[A.count] = total_b;
    A.ctl->total = total_i;
    A.ctl->groups = total_g;
    A.ctl->chunks_a = cut;
    A.ctl->units_b = total_b;
    A.ctl->unaligned = any_unaligned ? 1u : 0u;
    if (total_g > A.cap_groups) A.ctl->status = kStatusTooLong;
  }
}

// The multi-block batch planner (warp-chunk and stream kernels), three
// launches over tiles of 1024 strings, one thread per string and coalesced
// loads: it computes the plans that the one-block planner above computes,
// less the hybrid kernel's work list.

template <int L, int B = kLanes>
__device__ __forceinline__ unsigned long long plan_items(uint64_t N) {
  if (L == 0) return ((N + 7) >> 3) + 1;
  constexpr uint64_t CH = (uint64_t)(8 / B) << (3 * L);  // executions per item
  const uint64_t it = (N + CH - 1) / CH;
  return it ? it : 1ull;
}
template <int L>
__device__ __forceinline__ unsigned long long plan_groups(uint64_t N) {
  uint64_t g = 0;
  for (int lvl = (L == 0 ? 1 : L); lvl < kLevels; ++lvl) g += N >> (3 * lvl + 3);
  return g;
}

// 1: the work items and tree-group slots of every string of a tile, the
// tile's totals and whether it holds a string that is not 16-byte aligned.
// BIN: tree-group slots of the binary-tree ablation.
template <int W, int L, int B = kLanes, bool BIN = false>
__global__ void __launch_bounds__(1024) plan_tiles_kernel(const PlanArgs A) {
  constexpr uint64_t XB = Dims<W, B>::exec_bytes;
  __shared__ unsigned long long sh[32];
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long it = 0, gr = 0;
  bool un = false;
  if (i < A.count) {
    const uint64_t N = A.lens[i] / XB;
    it = plan_items<L, B>(N);
    gr = BIN ? bin_groups(N) : plan_groups<L>(N);
    un = (((uintptr_t)A.ptrs[i]) & 15u) != 0;
  }
  const int any_un = __syncthreads_or(un);
  unsigned long long ti, tg;
  block_scan(it, sh, &ti);
  block_scan(gr, sh, &tg);
  if (threadIdx.x == 0) {
    A.tile_items[blockIdx.x] = ti;
    A.tile_groups[blockIdx.x] = tg;
    A.tile_flags[blockIdx.x] = any_un ? 1u : 0u;
  }
}

// 2 (one block): the tiles' exclusive prefix sums, in place, the batch's
// totals, the capacity check and the alignment flag.
template <int W>
__global__ void __launch_bounds__(1024) plan_totals_kernel(const PlanArgs A) {
  __shared__ unsigned long long sh[32];
  unsigned long long base_i = 0, base_g = 0;
  int any_un = 0;
  for (unsigned t0 = 0; t0 < A.n_tiles; t0 += blockDim.x) {
    const unsigned t = t0 + threadIdx.x;
    const bool in = t < A.n_tiles;
    const unsigned long long vi = in ? A.tile_items[t] : 0, vg = in ? A.tile_groups[t] : 0;
    any_un |= __syncthreads_or(in && A.tile_flags[t] != 0);
    unsigned long long ti, tg;
    const unsigned long long ei = block_scan(vi, sh, &ti);
    const unsigned long long eg = block_scan(vg, sh, &tg);
    if (in) {
      A.tile_items[t] = base_i + ei;
      A.tile_groups[t] = base_g + eg;
    }
    base_i += ti;
    base_g += tg;
  }
  if (threadIdx.x == 0) {
    A.item0s[A.count] = base_i;
    A.ctl->total = base_i;
    A.ctl->groups = base_g;
    A.ctl->chunks_a = 0;
    A.ctl->units_b = 0;
    A.ctl->unaligned = any_un ? 1u : 0u;
    if (base_g > A.cap_groups || (A.item_str && base_i > A.cap_items)) A.ctl->status = kStatusTooLong;
  }
}

// 3: every string's plan, its first item and its first group slot.
template <int W, int L, int B = kLanes, bool BIN = false>
__global__ void __launch_bounds__(1024) plan_write_kernel(const PlanArgs A) {
  constexpr uint64_t XB = Dims<W, B>::exec_bytes;
  __shared__ unsigned long long sh[32];
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t len = 0, N = 0;
  unsigned long long it = 0, gr = 0;
  if (i < A.count) {
    len = A.lens[i];
    N = len / XB;
    it = plan_items<L, B>(N);
    gr = BIN ? bin_groups(N) : plan_groups<L>(N);
  }
  unsigned long long ti, tg;
  const unsigned long long ei = block_scan(it, sh, &ti) + A.tile_items[blockIdx.x];
  const unsigned long long eg = block_scan(gr, sh, &tg) + A.tile_groups[blockIdx.x];
  if (i < A.count) {
    StrPlan sp;
    sp.ptr = static_cast<const uint8_t *>(A.ptrs[i]);
    sp.len = len;
    sp.n_exec = N;
    sp.item0 = ei;
    sp.grp0 = eg;
    sp.n_items = (uint32_t)it;
    sp.pad = 0;
    sp.chunk0 = 0;
    sp.chunks_a = 0;
    sp.unitb0 = 0;
    A.plans[i] = sp;
    A.item0s[i] = ei;
  }
}

// 4: the string of every work item, so that a batch warp finds its string
// with one load instead of a search over item0s: one thread per item (grid
// stride), a binary search over the prefix sums.  (W only gives each width's
// table its own instance.)
template <int W>
__global__ void __launch_bounds__(256) plan_items_kernel(const PlanArgs A) {
  if (__ldcg(&A.ctl->status) != 0) return;
  const uint64_t total = __ldcg(&A.ctl->total);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += stride) {
    unsigned lo = 0, hi = A.count;  // item0s[lo] <= it < item0s[hi]
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) >> 1;
      if (A.item0s[mid] <= it) lo = mid; else hi = mid;
    }
    A.item_str[it] = lo;
  }
}

}  // namespace ht
