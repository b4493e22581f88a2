/*
 * halftime.h -- C ABI of libhalftime, a GB300 (sm_103a) implementation of
 * HalftimeHash (J. Apple, "HalftimeHash: Modern Hashing without 64-bit
 * Multipliers or Finite Fields", arXiv 2104.08865).
 *
 * The hash family maps a seed s and a byte string x to a 16, 24, 32 or
 * 40-byte digest H(s, x) (Section 1, problem statement; Section 2, output
 * widths).  Digests are k = width/8 little-endian 64-bit words.
 *
 * Conventions for every call:
 *   - Return value: HT_OK (0) or a negative HT_ERR_* code.  ht_last_error()
 *     gives a one-line description of the last error on the calling thread.
 *   - The caller owns every data, length, pointer-array and digest buffer.
 *     The library owns the opaque handles (ht_ctx, ht_server); release them
 *     with the matching *_destroy call.
 *   - "_dev" pointers are CUDA device pointers of the current device,
 *     "_host" pointers are host pointers.  ht_stream_t is a cudaStream_t
 *     (NULL = the legacy default stream).
 *   - Calls that take a stream only enqueue work on it and return without
 *     waiting; results are valid once the stream reaches that point.
 *   - A context keeps per-call scratch state on the device, so calls on one
 *     context must be ordered: issue them on one stream (or synchronise
 *     between streams).  Use one context per concurrent stream.
 *   - Lengths are bytes, 0 <= len < 2^64.
 */
#ifndef HALFTIME_H
#define HALFTIME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ht_stream_t; /* same type as cudaStream_t */
typedef struct ht_ctx ht_ctx;
typedef struct ht_server ht_server;
typedef struct ht_inc ht_inc;
typedef struct ht_table ht_table;

/* ---- status codes -------------------------------------------------------- */
#define HT_OK 0
#define HT_ERR_ARG -1      /* invalid argument (NULL pointer, size mismatch) */
#define HT_ERR_WIDTH -2    /* width not in {16, 24, 32, 40} (optionally | HT_BLOCK_256 or | HT_TREE_BINARY) */
#define HT_ERR_TOO_LONG -3 /* input or batch exceeds the context's capacity */
#define HT_ERR_CUDA -4     /* a CUDA runtime call failed (message has detail) */
#define HT_ERR_NOMEM -5    /* device or host allocation failed */
#define HT_ERR_BUDGET -6   /* request larger than the server's memory budget */
#define HT_ERR_TIMEOUT -7  /* a bounded wait ran out */
#define HT_ERR_BUSY -8     /* server queue full / ticket not finished */
#define HT_ERR_DEVICE -9   /* a kernel reported an error in the status word */

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to n bytes).  Returns the code of that error (HT_OK if none). */
int ht_last_error(char *buf, size_t n);

/* ---- seeds (Section 2 "input entropy"; Section 6.2 entropy budget) ----- */

/* Number of 64-bit seed words a width consumes.  The words are laid out as
 * E (e*w EHC hash keys), T (k*19*7 tree-node keys), F (k*19*8*8 final-NH
 * keys) and R (8*d*w + k Toeplitz tail keys): the budget of Section 6.2 for
 * 19 tree levels (enough for any length below 2^64), plus one tail key for
 * the length word.  Widths 16/24/32/40 give 2865/4245/5598/6897 words.
 * Returns 0 for an unsupported width. */
size_t ht_seed_words(int width_bytes);

/* ---- block size: 512-bit (default) or 256-bit blocks --------------------
 * Every width_bytes argument above and below may carry HT_BLOCK_256
 * (width_bytes | HT_BLOCK_256) to select blocks of b = 4 64-bit words instead
 * of the default b = 8 (Section 2, blocks of b words; Section 6.3, where the
 * 256-bit-block build is labelled "v3": the block size of processors
 * without 512-bit vectors).  With b = 4 an execution holds 8*4*d*w bytes
 * (672 / 672 / 480 bytes for widths 24 / 32 / 40 and 576 for width 16), the
 * tree runs over 4 lanes per output word, and the seed layout shrinks to
 * E, T, F = k*19*8*4 and R = 4*d*w + k words: 1577 / 2337 / 3082 / 3797
 * words for widths 16 / 24 / 32 / 40.  Digests differ from those of 8-word
 * blocks.  A context created with HT_BLOCK_256 serves ht_hash, ht_hash_host,
 * ht_hash_batch, ht_hash_batch_naive, the server and the digest table, with
 * the warp-chunk kernel only (ht_set_shape accepts kernel 1 with
 * chunk_levels 2; ht_autotune tunes its launch size); ht_inc_create,
 * ht_part_begin and ht_hash_noalloc reject it with HT_ERR_WIDTH. */
#define HT_BLOCK_256 0x100

/* ---- tree: the paper's T-hat (default) or the binary-tree ablation -------
 * A width_bytes argument may instead carry HT_TREE_BINARY (width_bytes |
 * HT_TREE_BINARY; not together with HT_BLOCK_256) to select the ablation
 * that the paper measures its tree against (Section 5.2, closing
 * paragraph: Badger's approach): per output word, Carter and Wegman's binary
 * tree T (Eq. algebraic-badger, Section 3.1) consumes the EHC outputs of all
 * executions and lanes whole (execution-major, lane-minor), with the
 * fan-out-2 NH node of Section 3.2 and one key per level; there is no final
 * NH over pending roots.  The Toeplitz tail with the length word is added as
 * in the default hash.  Seed layout: E (e*w words), 64 level keys per output
 * word, R (8*d*w + k): 295 / 390 / 458 / 472 words for widths 16 / 24 / 32 /
 * 40.  Digests differ from the default's.  A context created with
 * HT_TREE_BINARY serves ht_hash, ht_hash_host, ht_hash_batch,
 * ht_hash_batch_naive, the server and the digest table, with the warp-chunk
 * kernel and 64-execution items only (ht_set_shape accepts kernel 1 with
 * chunk_levels 2; ht_autotune tunes its launch size); ht_inc_create,
 * ht_part_begin and ht_hash_noalloc reject it with HT_ERR_WIDTH. */
#define HT_TREE_BINARY 0x200

/* Expands a 64-bit seed into the seed words of a width on the host: word i
 * is the i-th output of splitmix64 (Steele, Lea, Flood, OOPSLA 2014) started
 * at state seed64.  n_words must equal ht_seed_words(width_bytes).
 * Errors: HT_ERR_WIDTH, HT_ERR_ARG (NULL out_words or wrong n_words). */
int ht_seed_expand(uint64_t seed64, int width_bytes, uint64_t *out_words,
                   size_t n_words);

/* ---- context --------------------------------------------------------------
 * A context binds one width to one seed on the current CUDA device: it
 * uploads the seed words once, keeps the scratch memory of the tree stage
 * (per-group node accumulators and completion counters, Section 5.2), the
 * batch planner's buffers and the launch-shape cache of the autotuner.
 * seed_words_host: n_words host words (n_words = ht_seed_words(width)).
 * stream: the stream used for the uploads.
 * Errors: HT_ERR_WIDTH, HT_ERR_ARG, HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_ctx_create(int width_bytes, const uint64_t *seed_words_host,
                  size_t n_words, ht_stream_t stream, ht_ctx **out);
int ht_ctx_destroy(ht_ctx *ctx);

/* Replaces the context's seed (same width): uploads the new words on
 * `stream`; calls enqueued on that stream afterwards use them.  Errors:
 * HT_ERR_ARG (wrong n_words), HT_ERR_CUDA. */
int ht_ctx_rekey(ht_ctx *ctx, const uint64_t *seed_words_host, size_t n_words,
                 ht_stream_t stream);

/* Context flags.
 * HT_FLAG_OVERLAP_LAUNCHES: single-string launches of this context may start
 *   while the kernel before them in the stream is still finishing
 *   (programmatic dependent launch): each warp hashes its first chunk of the
 *   input before waiting for that kernel.  Safe only when the input of a call
 *   is never written by the kernel launched just before it (for example, not
 *   the digest buffer of the previous call); the context's own scratch is
 *   always protected.  Hides most of the fixed start and end cost of
 *   back-to-back hashes.  Default: off.
 * Errors: HT_ERR_ARG (unknown flag). */
#define HT_FLAG_OVERLAP_LAUNCHES 1u
int ht_ctx_set_flags(ht_ctx *ctx, unsigned flags);

/* Reserves device scratch so that ht_hash_batch can take up to max_strings
 * strings whose lengths add up to at most max_total_bytes (the default after
 * ht_ctx_create is 65536 strings and 16 GiB).  Synchronises the device.
 * Errors: HT_ERR_ARG, HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_ctx_reserve(ht_ctx *ctx, uint64_t max_total_bytes, size_t max_strings);

/* Waits for `stream`, then reads and clears the context's device status
 * word.  Returns HT_OK, or HT_ERR_TOO_LONG when a batch planned on the
 * device exceeded the reserved scratch (that batch's digests were not
 * written), HT_ERR_DEVICE when a bounded wait ran out or when the checked
 * build skipped an out-of-range access (the message names the buffer and
 * the index), or HT_ERR_CUDA.  After HT_ERR_DEVICE the digests of the calls
 * since the last status check are not valid, and the context's scratch
 * (tree groups, string sums, counters) is cleared before the call returns,
 * so the context hashes correctly again. */
int ht_ctx_status(ht_ctx *ctx, ht_stream_t stream);

/* Runs, on `stream`, the bounded wait that the stream kernel uses for its
 * shared-memory stages, on a stage that nothing fills, for `cycles` SM
 * clock cycles (1 .. 2^34): the wait runs out, the kernel reports it in the
 * context's status word and returns, and ht_ctx_status then gives
 * HT_ERR_DEVICE; the context stays usable.  For testing the timeout path.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_wait_probe(ht_ctx *ctx, uint64_t cycles, ht_stream_t stream);

/* ---- checked build ----------------------------------------------------------
 * The same sources compiled with -DHT_CHECK give libhalftime_check.so, a
 * debug library with the same entry points in which every global-memory
 * access of the warp-chunk kernels (single strings, batches, incremental
 * updates, both block sizes) is first checked against the extent of its
 * buffer (input string, seed region, tree-group scratch, per-string scratch,
 * digests, incremental stack).  An out-of-range index is never accessed: the
 * first one is recorded with its kind, the access is skipped (the digest is
 * then wrong), and ht_ctx_status / ht_inc_status report HT_ERR_DEVICE.  It
 * stands in for a memory checker where none can run; it is slower and is
 * not the product library. */
#define HT_BUILD_CHECKED 1u
/* Build flags of the loaded library: HT_BUILD_CHECKED for the checked build. */
unsigned ht_build_flags(void);
/* Runs the checked build's range check once on the device, on `index`
 * against `limit`, with no memory access at `index` (one thread; it tests
 * the recorder, not a kernel): with index >= limit, ht_ctx_status then
 * reports HT_ERR_DEVICE naming `index`.  In the normal build it does
 * nothing.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_check_probe(ht_ctx *ctx, uint64_t index, uint64_t limit, ht_stream_t stream);

/* ---- hashing ----------------------------------------------------------------
 * H(s, x) as in Section 5: generalized EHC over every 8*d*w-word execution
 * (Section 3.3, Section 4, Section 5.1), k f-ary NH tree hashes over the EHC
 * outputs with f = 8 (Section 3.1, Section 5.2, Eq. stack-construction), NH
 * over the pending tree roots plus a Toeplitz-keyed NH over the unread tail
 * and the length (Section 5.2, Section 6.1, Section 2). */

/* Hashes one device-resident string.  data_dev: len bytes (any alignment;
 * 16-byte aligned strings take the fast load path).  digest_dev: k words.
 * Errors: HT_ERR_ARG, HT_ERR_NOMEM (scratch growth failed), HT_ERR_CUDA. */
int ht_hash(ht_ctx *ctx, const void *data_dev, uint64_t len,
            uint64_t *digest_dev, ht_stream_t stream);

/* Hashes one string held in host memory (pinned memory gives full copy
 * speed; pageable memory works but is slower).  The string is copied to the
 * device in pieces on an internal copy stream while earlier pieces are
 * hashed; digest_host (k words) is written before the call returns, so this
 * call is synchronous.  Errors: as ht_hash, plus HT_ERR_NOMEM for the
 * staging buffer. */
int ht_hash_host(ht_ctx *ctx, const void *data_host, uint64_t len,
                 uint64_t *digest_host, ht_stream_t stream);

/* Hashes `count` device-resident strings in one persistent launch (the batch
 * form): ptrs_dev[i] / lens_dev[i] (device arrays) describe string i, and
 * digests_dev receives count*k words, string i at digests_dev + i*k.  A
 * device planner (one block for up to 1024 strings; else launches over
 * tiles of 1024 strings, then, from 16,384 strings, one that maps every work
 * item to its string) turns the lengths into a (string, chunk) work list; warps take chunks from an
 * atomic cursor; per-string completion counters finish each string's trees
 * and run its finaliser inside the same kernel (a string shorter than one
 * chunk is finished by the warp that hashes it).  The planner and the
 * kernel are replayed from a CUDA graph.  The batch must fit
 * the scratch reserved by ht_ctx_reserve: the planner checks this on the
 * device and, if it does not fit, writes no digests and records
 * HT_ERR_TOO_LONG for ht_ctx_status (the host cannot see device lengths).
 * Errors (host side): HT_ERR_ARG, HT_ERR_TOO_LONG (count above the reserve),
 * HT_ERR_CUDA. */
int ht_hash_batch(ht_ctx *ctx, const void *const *ptrs_dev,
                  const uint64_t *lens_dev, size_t count, uint64_t *digests_dev,
                  ht_stream_t stream);

/* The one-launch-per-string comparator of ht_hash_batch: ptrs_host and
 * lens_host are HOST arrays (of device pointers and lengths); string i is
 * hashed by its own ht_hash launch into digests_dev + i*k.  Same digests.
 * Errors: as ht_hash. */
int ht_hash_batch_naive(ht_ctx *ctx, const void *const *ptrs_host,
                        const uint64_t *lens_host, size_t count,
                        uint64_t *digests_dev, ht_stream_t stream);

/* ---- one string in parts (on several devices, or several launches) -------
 * A long string can be split at multiples of ht_part_granule(ctx) bytes (one
 * 64-execution chunk) and its parts hashed independently, each into the
 * "part state" of its own context (same width and seed; for example one
 * context per GPU).  A part state is an array of 64-bit words in which every
 * entry is a sum of contributions, so the states of all parts combine by
 * element-wise addition mod 2^64 — one all-reduce (sum, uint64) across
 * devices, or ht_part_merge on one device.  ht_finish_parts then completes
 * the tree groups whose children were split between parts and writes the
 * digest (Section 5.2 tree levels, Section 6.1 finaliser); the part that ends
 * the string has already added the tail, so finishing reads no input.
 * Sequence per context: ht_part_begin, ht_hash_part (any number of parts),
 * then either export the state (ht_part_state) or receive the others'
 * (ht_part_merge) and ht_finish_parts on one of them.  Calls on a context are
 * stream-ordered like the others. */

/* Bytes per split unit: parts start and end on multiples of this (0 for a
 * context of 256-bit blocks, which does not split strings). */
uint64_t ht_part_granule(ht_ctx *ctx);

/* Size in 64-bit words of the part state of a string of total_len bytes (0
 * for a context of 256-bit blocks). */
size_t ht_part_state_words(ht_ctx *ctx, uint64_t total_len);

/* Opens (and zeroes, on `stream`) the part state for a string of total_len
 * bytes.  state_dev: a device buffer of at least ht_part_state_words words
 * that the caller owns and keeps alive until ht_finish_parts (for example a
 * tensor it will all-reduce), or NULL for a buffer the context allocates.
 * Errors: HT_ERR_ARG (buffer too small), HT_ERR_WIDTH (a context of 256-bit
 * blocks), HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_part_begin(ht_ctx *ctx, uint64_t total_len, void *state_dev, size_t words,
                  ht_stream_t stream);

/* Hashes bytes [part_offset, part_offset + part_len) of the string into the
 * part state; part_dev points at the part's first byte (device).  part_offset
 * and, unless the part ends the string, part_len must be multiples of the
 * granule.  Errors: HT_ERR_ARG (no open state, misaligned or out-of-range
 * part), HT_ERR_CUDA. */
int ht_hash_part(ht_ctx *ctx, const void *part_dev, uint64_t part_offset,
                 uint64_t part_len, ht_stream_t stream);

/* The open part state: *state_dev (device array owned by the context) and
 * its size in 64-bit words, for exchanging it with other devices.
 * Errors: HT_ERR_ARG. */
int ht_part_state(ht_ctx *ctx, void **state_dev, size_t *words);

/* Adds another part state of the same string (a device array of `words`
 * 64-bit words on this context's device) into this context's state.
 * Errors: HT_ERR_ARG (size mismatch), HT_ERR_CUDA. */
int ht_part_merge(ht_ctx *ctx, const void *state_dev, size_t words,
                  ht_stream_t stream);

/* Completes the merged state and writes the k digest words to digest_dev;
 * closes the state.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_finish_parts(ht_ctx *ctx, uint64_t *digest_dev, ht_stream_t stream);

/* ---- incremental hashing: init / update / final ------------------------------
 * A string that arrives in pieces of any length, one after another, with its
 * total length unknown until the end (a file read in blocks, a network
 * stream, data larger than device memory).  The handle carries the string's
 * eager tree counter between calls (Section 5.2: for every level, the
 * pending nodes of its last, incomplete group, one value per tree and lane,
 * on a stack) plus a buffer of up to one 64-execution chunk of bytes.
 * Updates hash whole chunks straight from the caller's memory; only bytes
 * that straddle an update boundary are copied.  ht_inc_final hashes the
 * stack's pending nodes with their final keys, the buffered executions and
 * the tail (Section 6.1).  The digest equals ht_hash of the concatenation of
 * all pieces, for any way of cutting it.
 *   - A handle belongs to one context (its width and seed words) and must not
 *     outlive it; rekeying the context while a string is open gives a
 *     meaningless digest.
 *   - Calls on one handle are stream-ordered: issue them on one stream (or
 *     order the streams); one handle is not for concurrent host threads.
 *     Different handles are independent (each has its own scratch).
 *   - The state can be saved to host memory and restored into another
 *     handle of a context with the same width and seed words, in this or
 *     another process, to resume the string later.
 *   - After an update that returns an error the open string is lost (an
 *     update of more than 65536 chunks may have launched part of its work):
 *     ht_inc_init starts a new one, ht_inc_import resumes a saved state. */

/* Creates a handle (1.3 to 3.1 MB of device memory by width; host updates add
 * two staging slots of 1024 chunks) with an open, empty string.
 * Errors: HT_ERR_ARG, HT_ERR_WIDTH (a context of 256-bit blocks),
 * HT_ERR_CUDA. */
int ht_inc_create(ht_ctx *ctx, ht_inc **out);
int ht_inc_destroy(ht_inc *h);

/* Starts a new, empty string (clears the handle's scratch on `stream`).
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_inc_init(ht_inc *h, ht_stream_t stream);

/* Appends len bytes at data_dev (device, any alignment) to the string.
 * Asynchronous: data_dev must stay valid until `stream` reaches this point.
 * An update that completes a chunk is one kernel launch (two or more above
 * 65536 chunks): it reads the chunk begun by earlier updates from the
 * handle's buffer and from its own first bytes, and carries its own
 * remainder over into the handle's other buffer.  In a context with
 * HT_FLAG_OVERLAP_LAUNCHES it overlaps the kernel before it, under the same
 * rule as single-string launches (data_dev not written by the kernel
 * launched just before the call).  Errors: HT_ERR_ARG (no open string, NULL data), HT_ERR_TOO_LONG (total
 * length would exceed 2^64 - 1), HT_ERR_CUDA. */
int ht_inc_update(ht_inc *h, const void *data_dev, uint64_t len, ht_stream_t stream);

/* As ht_inc_update for bytes in HOST memory (pinned for full speed): whole
 * chunks are copied in pieces of 1024 chunks through two device slots on a
 * copy stream, each copy overlapping the hashing of the previous piece.
 * Returns once every byte has been consumed, so the caller may reuse its
 * buffer.  Errors: as ht_inc_update. */
int ht_inc_update_host(ht_inc *h, const void *data_host, uint64_t len, ht_stream_t stream);

/* Writes the k digest words of the string to digest_dev (device) and closes
 * it (ht_inc_init opens the next one).  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_inc_final(ht_inc *h, uint64_t *digest_dev, ht_stream_t stream);

/* Waits for `stream`, then reads and clears the handle's device status word
 * (its launches' own control block).  Returns HT_OK, or HT_ERR_DEVICE when
 * the checked build skipped an out-of-range access in one of the handle's
 * launches (see ht_build_flags), or HT_ERR_ARG, HT_ERR_CUDA. */
int ht_inc_status(ht_inc *h, ht_stream_t stream);

/* Bytes appended so far to the open string. */
uint64_t ht_inc_length(const ht_inc *h);

/* Bytes of one chunk (64 executions): updates whose lengths are multiples of
 * this, from a string start, copy nothing. */
uint64_t ht_inc_granule(const ht_inc *h);

/* Size in bytes of a saved state (header, stack, chunk buffer). */
size_t ht_inc_state_bytes(const ht_inc *h);

/* Saves the open string's state into state_host (n >= ht_inc_state_bytes
 * bytes, host memory); waits for `stream`.  The state records the width and
 * a fingerprint of the seed words.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_inc_export(const ht_inc *h, void *state_host, size_t n, ht_stream_t stream);

/* Replaces the handle's string by a saved state; waits for `stream`.
 * Errors: HT_ERR_ARG (short buffer, other width or seed words, corrupt
 * header), HT_ERR_CUDA. */
int ht_inc_import(ht_inc *h, const void *state_host, size_t n, ht_stream_t stream);

/* ---- long strings in a hash table by their digests ---------------------------
 * HalftimeHash is a universe-collapsing family (Section 1): it maps long
 * strings to short digests that a family made for short inputs can hash as
 * if they were the strings, and almost universality composes (the two
 * collision bounds add up: the composition lemma, Section 5.2).  An
 * ht_table keys strings by their digests on the device: entries are digests
 * numbered by insertion (ids 0, 1, ...); the first slot probed is the top
 * bits of a vector multiply-shift hash of the digest's 32-bit halves,
 *   h(x) = (a_0 + sum_i a_{i+1} x_i) mod 2^64,  x_0 = low half of word 0,
 *   x_1 = its high half, x_2 = low half of word 1, ...,
 * with keys a_0 .. a_2k the splitmix64 outputs of the table's seed (strongly
 * universal in its top l <= 33 bits); collisions probe linearly.  A slot
 * holds the smallest id of the entries with its digest, so inserting a batch
 * gives every entry's representative (deduplication by content) and a find
 * gives the id of an equal entry (a join).  Two different strings share a
 * digest with the probability bounded in Section 5 (about 2^-60 or less per
 * pair): then they are treated as equal.
 *   - The table holds at most max_entries entries and is at most half full
 *     (2^m >= 2 max_entries slots of 4 bytes, plus 8k bytes per entry).
 *   - Calls are stream-ordered like the context's; a table is for one stream
 *     (or ordered streams) and one host thread at a time. */

/* The 2k + 1 short-hash keys for a seed (host): n = 2 * width_bytes / 8 + 1.
 * Errors: HT_ERR_WIDTH, HT_ERR_ARG. */
int ht_short_hash_keys(uint64_t seed64, int width_bytes, uint64_t *keys_out, size_t n);

/* h(digest) above, on the host (the table computes the same on the device).
 * Errors: HT_ERR_WIDTH, HT_ERR_ARG. */
int ht_short_hash(const uint64_t *keys, int width_bytes, const uint64_t *digest, uint64_t *out);

/* Creates an empty table for digests of ctx's width (device memory as
 * above; ctx must outlive it).  max_entries: 1 .. 2^31.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_table_create(ht_ctx *ctx, uint64_t max_entries, uint64_t seed64, ht_table **out);
int ht_table_destroy(ht_table *t);

/* Removes every entry (on `stream`).  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_table_clear(ht_table *t, ht_stream_t stream);

/* Entries inserted so far; log2 of the slot count; the keys (2k + 1 words). */
uint64_t ht_table_entries(const ht_table *t);
int ht_table_slot_bits(const ht_table *t);
int ht_table_keys(const ht_table *t, uint64_t *keys_out, size_t n);

/* Inserts count digests (device, count*k words, for example ht_hash_batch's
 * output) as the next ids.  rep_dev (device, count uint32, or NULL):
 * rep_dev[i] = the smallest id, earlier insertions included, whose digest
 * equals digest i.  Errors: HT_ERR_ARG, HT_ERR_BUDGET (the table would
 * exceed max_entries; nothing is inserted), HT_ERR_CUDA. */
int ht_table_insert(ht_table *t, const uint64_t *digests_dev, size_t count, uint32_t *rep_dev,
                    ht_stream_t stream);

/* found_dev[i] (device uint32) = the smallest id whose digest equals query
 * digest i (device, count*k words), or 0xffffffff.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_table_find(ht_table *t, const uint64_t *digests_dev, size_t count, uint32_t *found_dev,
                  ht_stream_t stream);

/* Waits for `stream`; HT_ERR_BUDGET if a walk ever found no free slot (not
 * possible while the table is at most half full), else HT_OK. */
int ht_table_status(ht_table *t, ht_stream_t stream);

/* ---- hashing without allocation ---------------------------------------------
 * (The paper has no counterpart: this serves deployments, not the method.)
 * Some callers cannot allocate device memory: code running inside another
 * framework's allocator hooks (allocating there would re-enter the
 * allocator), processes whose device memory is held by another framework's
 * memory pool (an extra cudaMalloc fails or breaks that pool's accounting),
 * and latency-critical paths that cannot take the device synchronisation of
 * cudaMalloc/cudaFree.  They cannot create an ht_ctx.  ht_hash_noalloc hashes
 * one device-resident string with the warp-chunk kernel, using scratch that
 * the library reserves when it is loaded: one 8 MiB __device__ array,
 * present on every GPU that loads the library until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   - seed_words_host: the n_words = ht_seed_words(width_bytes) seed words on
 *     the host; they are copied into the array on `stream` (a copy from
 *     pageable memory is taken before the call returns; from pinned memory
 *     the words must stay unchanged until the stream reaches the copy).
 *   - data_dev / len / digest_dev / stream: as ht_hash (k digest words).
 *   - Limit: the tree scratch of the array holds 63107 / 42501 / 32039 /
 *     25710 node groups for widths 16 / 24 / 32 / 40, enough for strings of
 *     about 32 / 25 / 19 / 11 GB; longer strings return HT_ERR_TOO_LONG with
 *     no GPU work.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current) and loads the kernels this call
 *     launches for every width (with lazy module loading they would
 *     otherwise load, with driver-side allocations, at their first launch);
 *     make that first call before any stream capture.
 *   - Every call shares the one array and clears the parts it uses at the
 *     start, so calls that overlap on the GPU (other streams, other host
 *     threads) race and give wrong digests: order them.
 * Errors: HT_ERR_WIDTH (also for width_bytes | HT_BLOCK_256), HT_ERR_ARG,
 * HT_ERR_TOO_LONG, HT_ERR_CUDA. */
int ht_hash_noalloc(int width_bytes, const uint64_t *seed_words_host,
                    size_t n_words, const void *data_dev, uint64_t len,
                    uint64_t *digest_dev, ht_stream_t stream);

/* ---- launch shapes and autotuning ------------------------------------------
 * Four kernel families compute the same digests:
 *   kernel 0, the stream kernel: every warp owns a ring of `stages`
 *     shared-memory slots, each filled with one bulk copy (TMA) of 8
 *     executions, and hashes an equal, contiguous share of the work;
 *   kernel 1, the warp-chunk kernel (default): warps take chunks of 8^L
 *     executions from an atomic cursor and load them with 128-bit loads;
 *   kernel 2, the hybrid kernel: like kernel 1 with 64-execution chunks, but
 *     the last stretch of the launch is handed out as single 8-execution
 *     units;
 *   kernel 3, the block-chunk kernel (single strings only; the default below
 *     32 MiB): a block of eight warps takes a 64-execution chunk, one
 *     execution per thread, level 2 in shared memory; threads_per_block 256.
 * A shape also fixes the threads per block and blocks per SM.  The context
 * caches one shape per length bucket (bucket = floor(log2(len)), 0..63) and
 * one for batches. */
typedef struct ht_shape {
  int kernel;            /* 0: stream, 1: warp-chunk, 2: hybrid, 3: block-chunk */
  int chunk_levels;      /* warp-chunk kernel: L = 1, 2 or 3 */
  int stages;            /* stream kernel: shared-memory stages per warp, 2..8 */
  int threads_per_block; /* multiple of 32, at most 256 */
  int blocks_per_sm;     /* 1 .. 32; clamped to the occupancy limit */
} ht_shape;

/* The candidates are the warp-chunk kernel (chunk heights 1-3, 128 or 256
 * threads per block, 1-8 blocks per SM) and the block-chunk kernel (1-8
 * blocks per SM); the stream and hybrid families are selectable with
 * ht_set_shape but not tuned (on GB300 they won no length and no batch).
 * Times every candidate shape on `len`-byte strings in a device buffer
 * allocated and freed inside the call (at least 384 MiB, so that short
 * strings are timed from HBM, not from the L2 cache: each launch takes the
 * next copy) and stores the fastest in the bucket of len;
 * writes it to *best if best is not NULL.  Synchronous.  Errors: HT_ERR_ARG,
 * HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_autotune(ht_ctx *ctx, uint64_t len, ht_stream_t stream, ht_shape *best);

/* The same for batches (the persistent kernel of ht_hash_batch): times every
 * candidate batch shape -- the warp-chunk kernel's chunk height L
 * (executions per work item, 8^L: the parallelism a string gets), threads
 * per block and blocks per SM -- on the caller's own batch, and stores the
 * fastest as the
 * context's batch shape (the one ht_hash_batch and servers created from this
 * context use).  Arguments as for ht_hash_batch; digests_dev receives the
 * batch's digests (from the last run: the same for every shape).  A shape
 * whose planner finds that the batch does not fit the reserved scratch is
 * skipped.  Synchronous (several replays of the batch per candidate).
 * Errors: HT_ERR_ARG, HT_ERR_TOO_LONG (no shape fits), HT_ERR_CUDA. */
int ht_autotune_batch(ht_ctx *ctx, const void *const *ptrs_dev, const uint64_t *lens_dev,
                      size_t count, uint64_t *digests_dev, ht_stream_t stream,
                      ht_shape *best);

/* Reads / overrides the cached shape of the bucket of `len`
 * (len = UINT64_MAX selects the batch shape).  Errors: HT_ERR_ARG. */
int ht_get_shape(ht_ctx *ctx, uint64_t len, ht_shape *out);
int ht_set_shape(ht_ctx *ctx, uint64_t len, const ht_shape *shape);

/* Number of kernels this context has launched so far (planner and hash
 * kernels; graph replays count their kernel nodes). */
uint64_t ht_ctx_launches(ht_ctx *ctx);

/* ---- serving: continuous batching -------------------------------------------
 * A server admits hash requests as they arrive and keeps the GPU busy with
 * overlapping batches: a dispatcher thread forms a batch of the requests
 * that fit the free device memory (the budget) and a free stream slot,
 * stages pinned-host requests the GPU cannot read in place into a device
 * arena, and launches the batch on that slot's stream -- the batch graph,
 * or one single-string launch per request for a batch of at most eight
 * requests -- with the
 * batch's descriptors and digests in pinned host memory the GPU reads and
 * writes in place (else copied there and back); a completion thread
 * retires batches as their events fire, releases their memory and wakes
 * waiters.  Seeds and in-flight tree state stay on the device.  Every
 * request's arrival, launch and completion times are recorded (host
 * steady clock) for latency percentiles. */
typedef struct ht_server_opts {
  int n_streams;          /* concurrent batches in flight (default 8) */
  size_t max_batch;       /* requests per batch (default 4096) */
  size_t max_queue;       /* queued requests before submit says BUSY (default 1<<20) */
  uint64_t max_wait_us;   /* longest a request waits for batch-mates (default 0) */
  int pinned_mode;        /* pinned-host requests: 0 (default) = read in place by the
                             batch kernel when the GPU can address the memory (on
                             GB300 the coherent CPU-GPU link), else staged; the
                             batch descriptors and digests then stay in pinned host
                             memory too (no copies around a batch); 1 = always
                             staged, copied into a device arena first, with the
                             descriptors and digests copied as well */
} ht_server_opts;

typedef struct ht_server_stats_t {
  uint64_t submitted, completed, rejected, batches;
  uint64_t bytes_completed;
  double p50_us, p99_us, mean_us, max_us; /* arrival -> digest ready, completed requests */
  double wall_s;                          /* first arrival -> last completion */
} ht_server_stats_t;

/* Creates a server hashing with ctx's width and seed.  budget_bytes bounds
 * the device memory the server holds for request data in flight (the arena
 * is allocated here).  opts may be NULL for defaults.  The server owns its
 * own contexts and streams; ctx only provides width and seed and may be
 * destroyed afterwards.  Errors: HT_ERR_ARG, HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_server_create(ht_ctx *ctx, uint64_t budget_bytes,
                     const ht_server_opts *opts, ht_server **out);

/* Submits one request: `ptr` is either a device pointer (ptr_is_host_pinned
 * = 0; the data must stay valid until the request completes) or a host
 * pointer to pinned memory (ptr_is_host_pinned = 1; copied into the arena).
 * digest_host receives k words when the request completes.  *ticket
 * identifies the request.  Errors: HT_ERR_ARG, HT_ERR_BUDGET (len above the
 * budget: can never be admitted), HT_ERR_BUSY (queue full). */
int ht_server_submit(ht_server *srv, const void *ptr, uint64_t len,
                     int ptr_is_host_pinned, uint64_t *digest_host,
                     uint64_t *ticket);

/* *done = 1 once the request's digest is in digest_host.  Errors: HT_ERR_ARG
 * (unknown ticket). */
int ht_server_poll(ht_server *srv, uint64_t ticket, int *done);

/* Blocks until the request completes or timeout_us passes (HT_ERR_TIMEOUT).
 * A failed batch reports its error here (HT_ERR_CUDA / HT_ERR_DEVICE). */
int ht_server_wait(ht_server *srv, uint64_t ticket, uint64_t timeout_us);

/* Removes a request that is still queued (not yet launched); waiters on it
 * then get HT_ERR_ARG.  Returns HT_OK, HT_ERR_BUSY when the request was
 * already launched or finished, or HT_ERR_ARG (unknown ticket). */
int ht_server_cancel(ht_server *srv, uint64_t ticket);

/* Load replay: submits request i (ptrs[i], lens[i], pinned[i] as in
 * ht_server_submit; pinned may be NULL for all-device requests) at
 * arrival_us[i] microseconds after the call starts (non-decreasing offsets;
 * the submitting thread spins on the clock and submits every request that
 * is due at once), writing its digest to digests_host + i*k, then waits for
 * all of them (each wait bounded by timeout_us).  A request's latency is
 * counted from its scheduled arrival.  When the queue is full, due requests
 * wait in the replay loop.  *late_us (if not NULL) receives the largest delay
 * between a request's scheduled arrival and its submission.  Concurrent
 * ht_server_submit calls during a replay are not allowed (tickets of the
 * replay are consecutive).
 * Errors: HT_ERR_ARG, HT_ERR_BUDGET, HT_ERR_TIMEOUT, or the first failed
 * request's error. */
int ht_server_replay(ht_server *srv, const void *const *ptrs, const uint64_t *lens,
                     const int *pinned, const double *arrival_us, size_t n,
                     uint64_t *digests_host, uint64_t timeout_us, double *late_us);

/* Blocks until every submitted request has completed or timeout_us passes. */
int ht_server_drain(ht_server *srv, uint64_t timeout_us);

/* Statistics over completed requests since creation or the last reset. */
int ht_server_stats(ht_server *srv, ht_server_stats_t *out, int reset);

/* Per-request latencies (us, completion order) of completed requests since
 * the last reset: writes up to n values, returns how many were written. */
size_t ht_server_latencies(ht_server *srv, double *out_us, size_t n);

int ht_server_destroy(ht_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* HALFTIME_H */
