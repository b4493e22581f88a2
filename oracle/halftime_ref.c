/*
 * halftime_ref.c -- scalar CPU oracle for HalftimeHash (arXiv 2104.08865).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU
 * baseline of the benchmark.  The GPU library never uses this file.
 *
 * The hash follows the paper's three stages in order (Section 5):
 *   1. generalized EHC on each execution of b*d*w input words (Section 3.3,
 *      Section 4, Section 5.1): Encode with an erasure code of distance k,
 *      Hash every encoded word with NH, Combine with the k x e matrix T;
 *   2. k tree hashes over the EHC outputs (Section 3.1, Section 5.2,
 *      Eq. stack-construction) with the NH tree-node variant (Section 3.2);
 *   3. NH over the tree outputs plus a Toeplitz-keyed NH of the unread tail
 *      (Section 5.2, Section 6.1).
 *
 * Readings taken where the paper is silent or loose (all frozen):
 *  - Parameters: b = 8 words per block, f = 8, w = 3 for every width;
 *    (d, e, k) = (6,7,2), (7,9,3), (7,10,4), (5,9,5) for widths 16/24/32/40
 *    (Section 5.1 matrix shapes, Section 6.1 tuple for HalftimeHash24).
 *  - Codes: the paper's codes are not printed.  An item of w = 3 words is one
 *    GF(8) symbol, bit-sliced (word u holds the coefficient of x^u, GF(8) =
 *    GF(2)[x]/(x^3+x+1)), and each width uses a systematic MDS code: data
 *    items first, then parities P_r = sum_i A[i][r] * D_i.
 *  - Execution layout: word (blk, lane) of an execution at byte
 *    8*(blk*b + lane); item i of a lane = blocks i*w .. i*w+w-1 (Section 2).
 *  - NH pairs: the low and high 32-bit halves of a little-endian 64-bit word
 *    form one pair; seeds likewise (Section 3.2).
 *  - Tree: f-ary, merged eagerly, so the pending roots at level l are the
 *    base-f digit l of the execution count N, oldest first (Eq.
 *    stack-construction, generalized to fan-out f as in Section 6.1).
 *    A node over children x_0..x_{f-1} at level l is
 *    sum_{i<f-1} NH(x_i, S_T[t][l][i]) + x_{f-1} (Section 3.2 variant).
 *  - Final NH keys: S_F[t][l][j][lane] for the j-th pending root of level l;
 *    tail keys are Toeplitz: word m of component t uses R[t+m] (Section 6.1).
 *  - Tail: the N*b*d*w*8 bytes read by EHC are followed by the remaining
 *    bytes, zero padded to whole words, then one more word holding the byte
 *    length n (different-length strings are separated, Section 2).
 *  - Output t = final NH + tail NH, mod 2^64.
 */
#include "halftime_ref.h"

#include <stdlib.h>
#include <string.h>

#define REF_LEVELS 19 /* enough levels for any n < 2^64 bytes */
#define REF_W 3       /* words per item: one GF(8) symbol, bit-sliced */

/* ---- per-width constants, written from Section 5.1 ---------------------- */

/* Combine matrices T, rows t < k, columns c < e, as printed in Section 5.1. */
static const int T16[2][7] = {
    {1, 0, 1, 1, 2, 1, 4},
    {0, 1, 1, 2, 1, 4, 1},
};
static const int T24[3][9] = {
    {0, 0, 1, 4, 1, 1, 2, 2, 1},
    {1, 1, 0, 0, 1, 4, 1, 2, 2},
    {1, 4, 1, 1, 0, 0, 2, 1, 2},
};
static const int T32[4][10] = {
    {0, 0, 0, 1, 1, 4, 2, 4, 1, 1},
    {0, 1, 2, 0, 0, 1, 1, 2, 4, 1},
    {2, 0, 1, 0, 4, 0, 1, 1, 1, 1},
    {1, 1, 0, 1, 0, 0, 4, 1, 2, 8},
};
static const int T40[5][9] = {
    {1, 0, 0, 0, 0, 1, 1, 2, 4},
    {0, 1, 0, 0, 0, 1, 2, 1, 7},
    {0, 0, 1, 0, 0, 1, 3, 8, 5},
    {0, 0, 0, 1, 0, 1, 4, 9, 8},
    {0, 0, 0, 0, 1, 1, 5, 3, 9},
};

/* Parity coefficients A[i][r] over GF(8) (elements as 3-bit integers, bit v =
 * coefficient of x^v; alpha = x = 2).  Codes of the frozen reading:
 *   16: [7,6] single parity            P0 = sum D_i
 *   24: [9,7] P0 = sum D_i, P1 = sum alpha^i D_i
 *   32: [10,7] P_r = sum alpha^(r*i) D_i, r = 0,1,2
 *   40: [9,5] systematized doubly-extended Reed-Solomon code. */
static const unsigned char A16[6][1] = {{1}, {1}, {1}, {1}, {1}, {1}};
static const unsigned char A24[7][2] = {{1, 1}, {1, 2}, {1, 4}, {1, 3},
                                        {1, 6}, {1, 7}, {1, 5}};
static const unsigned char A32[7][3] = {{1, 1, 1}, {1, 2, 4}, {1, 4, 6},
                                        {1, 3, 5}, {1, 6, 2}, {1, 7, 3},
                                        {1, 5, 7}};
static const unsigned char A40[5][4] = {
    {1, 4, 1, 6}, {4, 5, 1, 1}, {1, 5, 5, 4}, {5, 1, 4, 1}, {4, 4, 5, 2}};

typedef struct {
  int d, e, k;
  const int *T;              /* k x e */
  const unsigned char *A;    /* d x (e-d) */
} width_spec;

static int get_spec(int width, width_spec *s) {
  switch (width) {
    case 16: s->d = 6; s->e = 7; s->k = 2; s->T = &T16[0][0]; s->A = &A16[0][0]; return 0;
    case 24: s->d = 7; s->e = 9; s->k = 3; s->T = &T24[0][0]; s->A = &A24[0][0]; return 0;
    case 32: s->d = 7; s->e = 10; s->k = 4; s->T = &T32[0][0]; s->A = &A32[0][0]; return 0;
    case 40: s->d = 5; s->e = 9; s->k = 5; s->T = &T40[0][0]; s->A = &A40[0][0]; return 0;
    default: return HTREF_ERR_WIDTH;
  }
}

int htref_params(int width, int *d, int *e, int *k, int *w, int *exec_bytes) {
  width_spec s;
  if (get_spec(width, &s)) return HTREF_ERR_WIDTH;
  *d = s.d; *e = s.e; *k = s.k; *w = REF_W;
  *exec_bytes = 8 * 8 * s.d * REF_W;
  return HTREF_OK;
}

/* ---- seed layout (Section 6.2 budget, 19 levels) ------------------------ */

typedef struct {
  size_t E, T, F, R, total;
} seed_layout;

static seed_layout layout_for(const width_spec *s, int b, int f) {
  seed_layout L;
  L.E = 0;
  L.T = L.E + (size_t)s->e * REF_W;
  L.F = L.T + (size_t)s->k * REF_LEVELS * (f - 1);
  L.R = L.F + (size_t)s->k * REF_LEVELS * f * b;
  L.total = L.R + (size_t)b * s->d * REF_W + s->k;
  return L;
}

size_t htref_seed_words_bf(int width, int b, int f) {
  width_spec s;
  if (get_spec(width, &s) || b < 1 || b > 8 || f < 2 || f > 8) return 0;
  return layout_for(&s, b, f).total;
}

size_t htref_seed_words(int width) { return htref_seed_words_bf(width, 8, 8); }

/* ---- splitmix64 (Steele, Lea, Flood 2014) ------------------------------- */

void htref_seed_expand(uint64_t seed64, uint64_t *out, size_t n) {
  uint64_t state = seed64;
  for (size_t i = 0; i < n; i++) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    out[i] = z ^ (z >> 31);
  }
}

/* ---- NH (Section 3.2) ---------------------------------------------------- */

uint64_t htref_nh_word(uint64_t x, uint64_t s) {
  uint32_t lo = (uint32_t)x + (uint32_t)s;               /* mod 2^32 */
  uint32_t hi = (uint32_t)(x >> 32) + (uint32_t)(s >> 32); /* mod 2^32 */
  return (uint64_t)lo * (uint64_t)hi;                      /* mod 2^64 */
}

/* ---- GF(8) arithmetic on bit-sliced items -------------------------------- */

/* c * D for a constant c in GF(8) and a bit-sliced item D (3 words): multiply
 * the polynomials, then reduce x^4 = x^2 + x and x^3 = x + 1. */
static void gf8_scale(unsigned c, const uint64_t *D, uint64_t *out) {
  uint64_t p[5] = {0, 0, 0, 0, 0};
  for (int v = 0; v < 3; v++)
    if ((c >> v) & 1)
      for (int u = 0; u < 3; u++) p[u + v] ^= D[u];
  p[2] ^= p[4];
  p[1] ^= p[4];
  p[1] ^= p[3];
  p[0] ^= p[3];
  out[0] = p[0];
  out[1] = p[1];
  out[2] = p[2];
}

static void encode_items(const width_spec *s, const uint64_t *items,
                         uint64_t *out) {
  int nparity = s->e - s->d;
  for (int i = 0; i < s->d; i++)
    for (int u = 0; u < REF_W; u++) out[i * REF_W + u] = items[i * REF_W + u];
  for (int r = 0; r < nparity; r++) {
    uint64_t acc[3] = {0, 0, 0};
    for (int i = 0; i < s->d; i++) {
      uint64_t t[3];
      gf8_scale(s->A[i * nparity + r], &items[i * REF_W], t);
      acc[0] ^= t[0];
      acc[1] ^= t[1];
      acc[2] ^= t[2];
    }
    for (int u = 0; u < REF_W; u++) out[(s->d + r) * REF_W + u] = acc[u];
  }
}

int htref_encode(int width, const uint64_t *items, uint64_t *out) {
  width_spec s;
  if (get_spec(width, &s)) return HTREF_ERR_WIDTH;
  encode_items(&s, items, out);
  return HTREF_OK;
}

/* ---- EHC: Encode, Hash, Combine (Section 3.3, Section 5.1) -------------- */

static uint64_t load_le64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

static void ehc_lane(const width_spec *s, int b, const uint64_t *E,
                     const uint8_t *exec, int lane, uint64_t *y) {
  uint64_t items[8 * REF_W], enc[10 * REF_W], h[10];
  /* gather the lane's d items (w blocks each) */
  for (int i = 0; i < s->d; i++)
    for (int u = 0; u < REF_W; u++) {
      int blk = i * REF_W + u;
      items[i * REF_W + u] = load_le64(exec + 8 * ((size_t)blk * b + lane));
    }
  /* Encode */
  encode_items(s, items, enc);
  /* Hash: NH of every encoded item under its own e*w seed words */
  for (int c = 0; c < s->e; c++) {
    h[c] = 0;
    for (int u = 0; u < REF_W; u++)
      h[c] += htref_nh_word(enc[c * REF_W + u], E[c * REF_W + u]);
  }
  /* Combine: y = T h over Z_{2^64} */
  for (int t = 0; t < s->k; t++) {
    uint64_t acc = 0;
    for (int c = 0; c < s->e; c++) acc += (uint64_t)s->T[t * s->e + c] * h[c];
    y[t] = acc;
  }
}

int htref_ehc(int width, int b, const uint64_t *seeds, const uint8_t *exec,
              int lane, uint64_t *y) {
  width_spec s;
  if (get_spec(width, &s)) return HTREF_ERR_WIDTH;
  if (b < 1 || b > 8 || lane < 0 || lane >= b) return HTREF_ERR_ARG;
  ehc_lane(&s, b, seeds, exec, lane, y);
  return HTREF_OK;
}

/* ---- tree node (Section 3.2 variant: last word added unhashed) ---------- */

static uint64_t tree_node(const uint64_t *children, int f,
                          const uint64_t *level_seeds) {
  uint64_t acc = 0;
  for (int i = 0; i < f - 1; i++) acc += htref_nh_word(children[i], level_seeds[i]);
  return acc + children[f - 1];
}

/* ---- streaming tree: eager base-f counter per (tree t, lane) ------------ */

typedef struct {
  uint64_t items[REF_LEVELS][8];
  int count[REF_LEVELS];
} tree_stack;

static void stack_push(tree_stack *st, int f, const uint64_t *Tseeds_t,
                       int level, uint64_t v) {
  for (;;) {
    st->items[level][st->count[level]++] = v;
    if (st->count[level] < f) return;
    v = tree_node(st->items[level], f, Tseeds_t + (size_t)level * (f - 1));
    st->count[level] = 0;
    level++;
  }
}

/* ---- recursive twin: complete f-ary tree over f^level EHC outputs ------- */

typedef struct {
  const width_spec *s;
  int b, f;
  const uint64_t *seeds;
  seed_layout L;
  const uint8_t *data;
  size_t exec_bytes;
} rec_ctx;

static uint64_t rec_tree(const rec_ctx *c, int t, int lane, int level,
                         uint64_t start) {
  if (level == 0) {
    uint64_t y[5];
    ehc_lane(c->s, c->b, c->seeds + c->L.E, c->data + start * c->exec_bytes,
             lane, y);
    return y[t];
  }
  uint64_t span = 1;
  for (int i = 0; i < level - 1; i++) span *= (uint64_t)c->f;
  uint64_t kids[8];
  for (int i = 0; i < c->f; i++)
    kids[i] = rec_tree(c, t, lane, level - 1, start + (uint64_t)i * span);
  const uint64_t *ts =
      c->seeds + c->L.T + ((size_t)t * REF_LEVELS + (level - 1)) * (c->f - 1);
  return tree_node(kids, c->f, ts);
}

/* ---- full hash ----------------------------------------------------------- */

int htref_hash_bf(int width, int b, int f, int recursive,
                  const uint64_t *seeds, size_t n_words, const uint8_t *data,
                  uint64_t len, uint64_t *digest, int *level_counts) {
  width_spec s;
  if (get_spec(width, &s)) return HTREF_ERR_WIDTH;
  if (b < 1 || b > 8 || f < 2 || f > 8) return HTREF_ERR_ARG;
  seed_layout L = layout_for(&s, b, f);
  if (n_words != L.total || seeds == NULL || digest == NULL) return HTREF_ERR_ARG;
  if (len > 0 && data == NULL) return HTREF_ERR_ARG;

  const size_t exec_words = (size_t)b * s.d * REF_W;
  const size_t exec_bytes = 8 * exec_words;
  const uint64_t N = len / exec_bytes; /* executions read by EHC */
  const int k = s.k;
  {
    /* the tree may not grow past REF_LEVELS levels (only reachable with the
     * small fan-outs of the debug parameters) */
    uint64_t cap = 1;
    int fits = 1;
    for (int l = 0; l < REF_LEVELS; l++) {
      if (cap > UINT64_MAX / (uint64_t)f) { fits = 0; break; }
      cap *= (uint64_t)f;
    }
    if (fits && N >= cap) return HTREF_ERR_ARG;
  }

  /* pending roots per (t, lane): roots[t][lane][level][j] */
  uint64_t(*roots)[8][REF_LEVELS][8] = calloc((size_t)k, sizeof(*roots));
  int counts[REF_LEVELS];
  if (!roots) return HTREF_ERR_ARG;

  if (!recursive) {
    tree_stack *st = calloc((size_t)k * b, sizeof(tree_stack));
    if (!st) { free(roots); return HTREF_ERR_ARG; }
    for (uint64_t x = 0; x < N; x++) {
      for (int lane = 0; lane < b; lane++) {
        uint64_t y[5];
        ehc_lane(&s, b, seeds + L.E, data + x * exec_bytes, lane, y);
        for (int t = 0; t < k; t++)
          stack_push(&st[t * b + lane], f,
                     seeds + L.T + (size_t)t * REF_LEVELS * (f - 1), 0, y[t]);
      }
    }
    for (int t = 0; t < k; t++)
      for (int lane = 0; lane < b; lane++)
        for (int l = 0; l < REF_LEVELS; l++)
          for (int j = 0; j < st[t * b + lane].count[l]; j++)
            roots[t][lane][l][j] = st[t * b + lane].items[l][j];
    for (int l = 0; l < REF_LEVELS; l++) counts[l] = st[0].count[l];
    free(st);
  } else {
    /* digits of N in base f, highest level first; each digit is a run of
     * complete trees taken from the front of the remaining input */
    rec_ctx c = {&s, b, f, seeds, L, data, exec_bytes};
    uint64_t pos = 0;
    for (int l = REF_LEVELS - 1; l >= 0; l--) {
      uint64_t span = 1;
      int overflow = 0;
      for (int i = 0; i < l; i++) {
        if (span > N / (uint64_t)f) { overflow = 1; break; }
        span *= (uint64_t)f;
      }
      counts[l] = 0;
      if (overflow) continue;
      while (N - pos >= span) {
        int j = counts[l]++;
        for (int t = 0; t < k; t++)
          for (int lane = 0; lane < b; lane++)
            roots[t][lane][l][j] = rec_tree(&c, t, lane, l, pos);
        pos += span;
      }
    }
  }
  if (level_counts)
    for (int l = 0; l < REF_LEVELS; l++) level_counts[l] = counts[l];

  /* Final NH over the pending roots (Section 5.2) */
  for (int t = 0; t < k; t++) {
    uint64_t acc = 0;
    for (int l = 0; l < REF_LEVELS; l++)
      for (int j = 0; j < counts[l]; j++)
        for (int lane = 0; lane < b; lane++) {
          size_t fi = L.F + (((size_t)t * REF_LEVELS + l) * f + j) * b + lane;
          acc += htref_nh_word(roots[t][lane][l][j], seeds[fi]);
        }
    digest[t] = acc;
  }
  free(roots);

  /* Tail NH with Toeplitz keys (Section 6.1), length word appended */
  const uint64_t tail_start = N * exec_bytes;
  const uint64_t tail_len = len - tail_start;
  const uint64_t M = (tail_len + 7) / 8;
  for (uint64_t m = 0; m <= M; m++) {
    uint64_t word;
    if (m == M) {
      word = len;
    } else {
      uint8_t buf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      uint64_t avail = tail_len - 8 * m;
      memcpy(buf, data + tail_start + 8 * m, avail < 8 ? (size_t)avail : 8);
      word = load_le64(buf);
    }
    for (int t = 0; t < k; t++) digest[t] += htref_nh_word(word, seeds[L.R + t + m]);
  }
  return HTREF_OK;
}

int htref_hash(int width, const uint64_t *seeds, size_t n_words,
               const uint8_t *data, uint64_t len, uint64_t *digest) {
  return htref_hash_bf(width, 8, 8, 0, seeds, n_words, data, len, digest, NULL);
}

/* ---- ablation: Badger's binary tree without a final NH (Section 5.2) ----- */

#define REF_BADGER_LEVELS 64 /* T keys per tree: a node spans < 2^64 leaves */

size_t htref_seed_words_badger(int width, int b) {
  width_spec s;
  if (get_spec(width, &s) || b < 1 || b > 8) return 0;
  return (size_t)s.e * REF_W + (size_t)s.k * REF_BADGER_LEVELS +
         (size_t)b * s.d * REF_W + s.k;
}

/* ceil(lg n) for n >= 1 */
static int ceil_lg(uint64_t n) {
  int m = 0;
  while (m < 64 && ((uint64_t)1 << m) < n) m++;
  return m;
}

/* Eq. algebraic-badger over the leaves s[0, n), n >= 1: a single leaf is
 * itself; a longer span splits after its first 2^(ceil(lg n) - 1) leaves and
 * H(k_i, left, right) = NH(left, k_i) + right joins the two halves, with
 * i = ceil(lg n) - 1. */
static uint64_t badger_T(const uint64_t *keys, const uint64_t *s, uint64_t n) {
  if (n == 1) return s[0];
  const int i = ceil_lg(n) - 1;
  const uint64_t half = (uint64_t)1 << i;
  return htref_nh_word(badger_T(keys, s, half), keys[i]) +
         badger_T(keys, s + half, n - half);
}

int htref_hash_badger(int width, int b, const uint64_t *seeds, size_t n_words,
                      const uint8_t *data, uint64_t len, uint64_t *digest) {
  width_spec s;
  if (get_spec(width, &s)) return HTREF_ERR_WIDTH;
  if (b < 1 || b > 8) return HTREF_ERR_ARG;
  if (n_words != htref_seed_words_badger(width, b) || seeds == NULL || digest == NULL)
    return HTREF_ERR_ARG;
  if (len > 0 && data == NULL) return HTREF_ERR_ARG;
  const int k = s.k;
  const size_t off_T = (size_t)s.e * REF_W;
  const size_t off_R = off_T + (size_t)k * REF_BADGER_LEVELS;
  const size_t exec_bytes = 8 * (size_t)b * s.d * REF_W;
  const uint64_t N = len / exec_bytes;
  const uint64_t n_leaves = N * (uint64_t)b;

  /* EHC of every execution and lane: leaf x*b + lane of tree t */
  uint64_t *leaves = NULL;
  if (n_leaves) {
    leaves = malloc((size_t)k * n_leaves * sizeof(uint64_t));
    if (!leaves) return HTREF_ERR_ARG;
    for (uint64_t x = 0; x < N; x++)
      for (int lane = 0; lane < b; lane++) {
        uint64_t y[5];
        ehc_lane(&s, b, seeds, data + x * exec_bytes, lane, y);
        for (int t = 0; t < k; t++) leaves[(size_t)t * n_leaves + x * b + lane] = y[t];
      }
  }
  for (int t = 0; t < k; t++)
    digest[t] = n_leaves ? badger_T(seeds + off_T + (size_t)t * REF_BADGER_LEVELS,
                                    leaves + (size_t)t * n_leaves, n_leaves)
                         : 0;
  free(leaves);

  /* Tail NH with Toeplitz keys (Section 6.1), length word appended */
  const uint64_t tail_start = N * exec_bytes;
  const uint64_t tail_len = len - tail_start;
  const uint64_t M = (tail_len + 7) / 8;
  for (uint64_t m = 0; m <= M; m++) {
    uint64_t word;
    if (m == M) {
      word = len;
    } else {
      uint8_t buf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      uint64_t avail = tail_len - 8 * m;
      memcpy(buf, data + tail_start + 8 * m, avail < 8 ? (size_t)avail : 8);
      word = load_le64(buf);
    }
    for (int t = 0; t < k; t++) digest[t] += htref_nh_word(word, seeds[off_R + t + m]);
  }
  return HTREF_OK;
}
