// ht_check.cuh -- bounds checks of the checked build (compiled with
// -DHT_CHECK into libhalftime_check.so; compute-sanitizer is not available
// everywhere, so the library can check itself).
//
// In a checked build every global-memory access of the kernels (all four
// families; a bulk copy by its whole range) is preceded by a check of its
// index against the extent of its buffer: the input string, a seed region,
// the tree-group scratch, the per-string scratch, the digests, the
// incremental stack and chunk buffers.  An index outside its buffer
// is not accessed: the check records the first such (kind, index) in the
// launch's control block, sets a status bit, and the access is skipped, so
// the kernel neither faults nor traps; the host reports it as
// HT_ERR_DEVICE (ht_ctx_status, ht_inc_status).  In the normal build each
// check is the constant true and compiles away.
#pragma once

#include "ht_internal.h"

namespace ht {

constexpr unsigned int kStatusBounds = 4;  // checked build: an out-of-range access was skipped

// What a check guards (Ctl::bad_kind).
enum CheckKind : unsigned int {
  kChkInput = 1,   // input bytes: an execution or a tail word past the string
  kChkSeedT = 2,   // tree-node keys (T region)
  kChkSeedF = 3,   // final-NH keys (F region)
  kChkSeedR = 4,   // Toeplitz tail keys (R region)
  kChkGroup = 5,   // tree-group slot (accumulators and arrival counters)
  kChkString = 6,  // per-string scratch (pending-root sums, completion counts)
  kChkDigest = 7,  // digest row
  kChkStack = 8,   // incremental stack slot
  kChkIncBuf = 9,  // incremental chunk buffer (the buffered bytes, the remainder carried over)
};

#ifdef HT_CHECK
static __device__ __noinline__ bool check_failed(Ctl *ctl, unsigned int kind, uint64_t index) {
  if (atomicCAS(&ctl->bad_kind, 0u, kind) == 0u) ctl->bad_index = index;
  atomicOr(&ctl->status, kStatusBounds);
  return false;
}
static __device__ __forceinline__ bool in_range(Ctl *ctl, unsigned int kind, uint64_t index, uint64_t limit) {
  return index < limit ? true : check_failed(ctl, kind, index);
}
// true when index < limit; otherwise records (kind, index) and gives false
#define HT_IN_RANGE(P, kind, index, limit) \
  (::ht::in_range((P).scr.ctl, (kind), (uint64_t)(index), (uint64_t)(limit)))
constexpr bool kChecked = true;
#else
#define HT_IN_RANGE(P, kind, index, limit) true
constexpr bool kChecked = false;
#endif

}  // namespace ht
