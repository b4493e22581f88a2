/*
 * halftime_testing.h -- host-only test hooks of libhalftime.
 *
 * The paper has no serving system; these hooks exist so that the serving
 * loop's host logic (admission by budget, queue limits, timeouts,
 * cancellation, error propagation) can be tested on machines without a GPU
 * and without ever making a GPU fail.  A fake server runs the same
 * dispatcher and completion threads as ht_server_create, but its "device"
 * is a host timer: a batch completes `batch_delay_us` after launch, digests
 * are written as zeros, and batch number `fail_batch` (0-based, -1 = never)
 * completes with HT_ERR_CUDA instead.
 */
#ifndef HALFTIME_TESTING_H
#define HALFTIME_TESTING_H

#include "halftime.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Creates a fake server for `width_bytes` (16/24/32/40): no CUDA calls are
 * made.  budget_bytes, opts: as ht_server_create.  Errors: HT_ERR_WIDTH,
 * HT_ERR_ARG. */
int ht_server_create_fake(int width_bytes, uint64_t budget_bytes,
                          const ht_server_opts *opts, uint64_t batch_delay_us,
                          int64_t fail_batch, ht_server **out);

/* Sets the limit, in SM clock cycles, of the stream kernel's waits for its
 * shared-memory stages on this context (0: the default, about a second;
 * at most 2^34).  The wait that lets a warp's copies in flight land before
 * it exits keeps the default.  With a limit of a few cycles the first stage
 * wait runs out while its copy is still in flight: the kernel reports
 * HT_ERR_DEVICE through ht_ctx_status, which also clears the context's
 * scratch, and the context hashes correctly afterwards.  Errors:
 * HT_ERR_ARG. */
int ht_testing_set_wait_cycles(ht_ctx *ctx, uint64_t cycles);

#ifdef __cplusplus
}
#endif

#endif /* HALFTIME_TESTING_H */
