/*
 * halftime_ref.h -- scalar CPU oracle for HalftimeHash (arXiv 2104.08865).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that tests, the smoke
 * check and the CPU-baseline leg of the benchmark can compare the GPU library
 * against a plain, slow, obviously correct implementation.  The product
 * (the CUDA library and its Python binding) never links, loads or calls it,
 * and it shares no source with the product.
 *
 * Every function follows the paper step by step; the readings taken where the
 * paper is silent are listed at the top of halftime_ref.c.
 *
 * Parity status: every function here is pinned by tests against facts the
 * paper or mathematics fixes (combine matrices and their 2-adic minors, code
 * distance by exhaustive enumeration, published splitmix64 outputs, the
 * paper's seed-size figures, tree-shape digit sums, a recursive twin,
 * brute-force evaluation of the paper's recursive equations at b=1, f=2, NH
 * closed forms, Toeplitz shift).  Absolute digest values of the full b=8, f=8
 * hash have no published test vectors: that end-to-end value is "parity
 * unpinned" beyond the structural pins above.
 */
#ifndef HALFTIME_REF_H
#define HALFTIME_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (negative = error). */
#define HTREF_OK 0
#define HTREF_ERR_ARG -1
#define HTREF_ERR_WIDTH -2

/* Number of 64-bit seed words the hash of width `width_bytes` (16/24/32/40)
 * consumes with block size b and fan-out f (the library default is b=8, f=8).
 * Layout (Section 6.1, Section 6.2 entropy budget, with 19 tree levels):
 *   E: e*w words, T: k*19*(f-1), F: k*19*f*b, R: b*d*w + k.
 * Returns 0 for an unknown width. */
size_t htref_seed_words(int width_bytes);
size_t htref_seed_words_bf(int width_bytes, int b, int f);

/* Seed word i = i-th output of splitmix64 started at state seed64
 * (Steele, Lea, Flood, OOPSLA 2014). */
void htref_seed_expand(uint64_t seed64, uint64_t *out_words, size_t n_words);

/* Encode step of EHC for one lane (Section 3.3, Section 5.1): `items` holds
 * d items of w=3 words (item-major), `out` receives e items of 3 words: the
 * d data items followed by the e-d parity items of the GF(8) code. */
int htref_encode(int width_bytes, const uint64_t *items, uint64_t *out);

/* One EHC execution for one lane: reads the execution's b*d*w words from
 * `exec_bytes` (little-endian, word (blk, lane) at byte 8*(blk*b + lane)),
 * encodes, hashes with NH under the E seed region and combines with the
 * paper's matrix T.  Writes k words to y_out. */
int htref_ehc(int width_bytes, int b, const uint64_t *seed_words,
              const uint8_t *exec_bytes, int lane, uint64_t *y_out);

/* NH of one 64-bit word against one seed word: (lo+s.lo)*(hi+s.hi) mod 2^64
 * with the two sums mod 2^32 (Section 3.2). */
uint64_t htref_nh_word(uint64_t x, uint64_t s);

/* Full hash, b=8, f=8.  `seed_words` must hold htref_seed_words(width)
 * words.  Writes k = width/8 little-endian words to `digest`. */
int htref_hash(int width_bytes, const uint64_t *seed_words, size_t n_words,
               const uint8_t *data, uint64_t len, uint64_t *digest);

/* Same hash, general block size b (1..8) and fan-out f (2..8).  When
 * `recursive` is nonzero the tree stage is evaluated by the recursive
 * definition (complete f-ary trees per base-f digit of the execution count)
 * instead of the streaming counter.  When `level_counts` is not NULL it
 * receives, per level 0..18, the number of pending roots left by the
 * streaming counter (tree t=0, lane 0). */
int htref_hash_bf(int width_bytes, int b, int f, int recursive,
                  const uint64_t *seed_words, size_t n_words,
                  const uint8_t *data, uint64_t len, uint64_t *digest,
                  int *level_counts);

/* The ablation of Section 5.2: Badger's binary tree T (Eq. algebraic-badger)
 * consumes the EHC outputs whole, with no pending roots and no final NH.
 * Per tree t the leaves are the EHC outputs y_t of every execution and lane,
 * execution-major and lane-minor (leaf x*b + lane); T splits a span of n > 1
 * leaves at 2^(ceil(lg n) - 1) and joins the halves with the fan-out-2 node
 * H(k_i, x, y) = NH(x, k_i) + y, i = ceil(lg n) - 1 (Section 3.1, Section 3.2
 * node variant).  Output t = T_t (0 without leaves) + the Toeplitz tail NH with
 * the length word, as in the default hash.
 * Seed layout: E: e*w words, T: k*64 level keys (key i of tree t at
 * e*w + 64*t + i), R: b*d*w + k. */
size_t htref_seed_words_badger(int width_bytes, int b);
int htref_hash_badger(int width_bytes, int b, const uint64_t *seed_words,
                      size_t n_words, const uint8_t *data, uint64_t len,
                      uint64_t *digest);

/* Parameters of a width: fills {d, e, k, w, exec_bytes(b=8)}. */
int htref_params(int width_bytes, int *d, int *e, int *k, int *w,
                 int *exec_bytes);

#ifdef __cplusplus
}
#endif

#endif
