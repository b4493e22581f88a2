// ht_spec.cuh -- compile-time description of the four HalftimeHash widths
// for the GPU path (arXiv 2104.08865, Section 5.1 and Section 6.1).
//
// Per width: d data items and e encoded items of w = 3 words per EHC lane, k
// output words, the paper's k x e combine matrix T (Section 5.1), and the
// parity coefficients of the erasure code.  An item of three 64-bit words is
// read as 64 independent GF(8) symbols, word u holding the x^u coefficient
// (GF(8) = GF(2)[x]/(x^3+x+1)), so every code below is pure XOR work:
//   16: one parity  P0 = sum D_i                            (distance 2)
//   24: P0 = sum D_i, P1 = sum a^i D_i                      (distance 3)
//   32: P_r = sum a^(r i) D_i, r = 0..2                      (distance 4)
//   40: systematized doubly-extended Reed-Solomon [9,5]     (distance 5)
// with a = x the primitive element.
#pragma once

#include <cstdint>

namespace ht {

constexpr int kLevels = 19;   // tree levels: 8^19 executions > 2^64 bytes
constexpr int kLanes = 8;     // b: 64-bit words per block (Section 6.1)
constexpr int kFan = 8;       // f: tree fan-out (Section 6.1)
constexpr int kItemWords = 3; // w: words per encoded item (Section 6.1)
constexpr int kMaxK = 5;
constexpr int kMaxEW = 30;    // max e*w

// Multiplication in GF(8) with reduction x^4 -> x^2 + x, x^3 -> x + 1.
__host__ __device__ constexpr unsigned gf8_mul(unsigned a, unsigned b) {
  unsigned r = 0;
  for (int i = 0; i < 3; ++i)
    if ((b >> i) & 1u) r ^= a << i;
  if (r & 16u) r ^= 0x16u;  // x^4 + x^2 + x
  if (r & 8u) r ^= 0xBu;    // x^3 + x + 1
  return r;
}

// Does input plane u of an item feed output plane v of c * item?
__host__ __device__ constexpr bool gf8_feeds(unsigned c, int u, int v) {
  return ((gf8_mul(c, 1u << u) >> v) & 1u) != 0;
}

template <int W>
struct Spec;

template <>
struct Spec<16> {
  static constexpr int d = 6, e = 7, k = 2;
  __host__ __device__ static constexpr int T(int t, int c) {
    const int m[2][7] = {{1, 0, 1, 1, 2, 1, 4}, {0, 1, 1, 2, 1, 4, 1}};
    return m[t][c];
  }
  __host__ __device__ static constexpr unsigned A(int /*i*/, int /*r*/) { return 1u; }
};

template <>
struct Spec<24> {
  static constexpr int d = 7, e = 9, k = 3;
  __host__ __device__ static constexpr int T(int t, int c) {
    const int m[3][9] = {{0, 0, 1, 4, 1, 1, 2, 2, 1},
                         {1, 1, 0, 0, 1, 4, 1, 2, 2},
                         {1, 4, 1, 1, 0, 0, 2, 1, 2}};
    return m[t][c];
  }
  __host__ __device__ static constexpr unsigned A(int i, int r) {
    // column r = 0: all ones; column r = 1: a^i
    const unsigned pw[7] = {1, 2, 4, 3, 6, 7, 5};
    return r == 0 ? 1u : pw[i];
  }
};

template <>
struct Spec<32> {
  static constexpr int d = 7, e = 10, k = 4;
  __host__ __device__ static constexpr int T(int t, int c) {
    const int m[4][10] = {{0, 0, 0, 1, 1, 4, 2, 4, 1, 1},
                          {0, 1, 2, 0, 0, 1, 1, 2, 4, 1},
                          {2, 0, 1, 0, 4, 0, 1, 1, 1, 1},
                          {1, 1, 0, 1, 0, 0, 4, 1, 2, 8}};
    return m[t][c];
  }
  __host__ __device__ static constexpr unsigned A(int i, int r) {
    const unsigned pw[7] = {1, 2, 4, 3, 6, 7, 5};
    return pw[(r * i) % 7];
  }
};

template <>
struct Spec<40> {
  static constexpr int d = 5, e = 9, k = 5;
  __host__ __device__ static constexpr int T(int t, int c) {
    const int m[5][9] = {{1, 0, 0, 0, 0, 1, 1, 2, 4},
                         {0, 1, 0, 0, 0, 1, 2, 1, 7},
                         {0, 0, 1, 0, 0, 1, 3, 8, 5},
                         {0, 0, 0, 1, 0, 1, 4, 9, 8},
                         {0, 0, 0, 0, 1, 1, 5, 3, 9}};
    return m[t][c];
  }
  __host__ __device__ static constexpr unsigned A(int i, int r) {
    const unsigned m[5][4] = {{1, 4, 1, 6}, {4, 5, 1, 1}, {1, 5, 5, 4},
                              {5, 1, 4, 1}, {4, 4, 5, 2}};
    return m[i][r];
  }
};

// Derived sizes of a width with B words per block: B = 8 (512-bit blocks,
// the paper's default) or B = 4 (256-bit blocks, the variant the paper labels
// "v3" in Section 6.3).  B fixes the execution size and the sizes of the
// final-NH and tail key regions.
template <int W, int B = kLanes>
struct Dims {
  static_assert(B == 8 || B == 4, "blocks of 8 or 4 words");
  static constexpr int d = Spec<W>::d, e = Spec<W>::e, k = Spec<W>::k;
  static constexpr int dw = d * kItemWords;              // data words per lane
  static constexpr int ew = e * kItemWords;              // seed words of E
  static constexpr int exec_bytes = 8 * B * dw;          // one EHC execution
  // seed regions, in words
  static constexpr int off_T = ew;
  static constexpr int off_F = off_T + k * kLevels * (kFan - 1);
  static constexpr int off_R = off_F + k * kLevels * kFan * B;
  static constexpr int n_seed = off_R + B * dw + k;
};

// Seed layout of the binary-tree ablation (Badger's approach, Section 5.2):
// the EHC keys E (e*w words), then 64 level keys per tree (key h of tree t at
// off_T + 64 t + h; a binary node spans fewer than 2^64 leaves), then the
// Toeplitz tail keys; no final-NH region.  512-bit blocks.
constexpr int kBinLevels = 64;
template <int W>
struct BinDims {
  static constexpr int k = Spec<W>::k;
  static constexpr int off_T = Dims<W>::ew;
  static constexpr int off_R = off_T + k * kBinLevels;
  static constexpr int n_seed = off_R + kLanes * Dims<W>::dw + k;
};

// Tree-group slots of a string of N executions under the binary-tree
// ablation: one per pair of complete nodes at every height h >= 9 (above a
// 64-execution work item), where height h holds N >> (h - 3) complete nodes.
__host__ __device__ inline unsigned long long bin_groups(uint64_t N) {
  unsigned long long g = 0;
  for (int j = 6; j < 64; ++j) g += (N >> j) >> 1;
  return g;
}

}  // namespace ht
