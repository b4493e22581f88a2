// ht_table.cu -- long strings in a hash table by their digests.
//
// HalftimeHash is a universe-collapsing family (Section 1): it maps long
// strings to short digests, which a family made for short inputs can then
// hash as if they were the strings; almost universality composes, the two
// collision bounds adding up (the composition lemma, Section 5.2).  This
// table does that on the GPU: entries are digests (k words, numbered by
// insertion), the first slot probed is the top bits of a vector
// multiply-shift hash of the digest's 32-bit halves,
//     h(x) = (a_0 + sum_i a_{i+1} x_i) mod 2^64,
// strongly universal in its top l <= 33 bits for uniform 64-bit keys
// (Dietzfelbinger et al. 1997; vector form after Thorup 2015), and
// collisions probe linearly.  A slot holds the smallest id of the entries
// with its digest, so inserting a batch yields each entry's representative
// (deduplication by content) and finding a digest yields the id of an equal
// entry (a join).
//
// Layout: the digests of all entries, row e = entry e (k words), and the
// slots, 2^m 32-bit entry ids (0xffffffff: empty), at most half full.  An
// insertion first copies the batch's digests into their rows; the insert
// kernel then claims slots with compare-and-swap and keeps the smallest id
// of equal digests with atomic min; a find walks from the first slot to an
// equal digest or an empty slot.  Every walk ends: the table is never more
// than half full, and the walk length is bounded by the slot count anyway
// (a status word reports a walk that hit the bound, which cannot happen
// while the occupancy limit holds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "halftime.h"
#include "ht_internal.h"
#include "ht_runtime.h"

using namespace ht;

namespace {

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kMaxKeys = 11;  // 2k + 1 for k <= 5

struct TableArgs {
  unsigned long long keys[kMaxKeys];
  const unsigned long long *rows;   // digests of the entries
  unsigned int *slots;
  unsigned int *status;
  const unsigned long long *query;  // insert: rows of the new entries; find: the queries
  unsigned int *out;                // find: the ids found
  unsigned long long count;
  unsigned int base;                // insert: id of the first new entry
  int shift;                        // 64 - m
  unsigned long long mask;          // 2^m - 1
};

template <int K>
__device__ __forceinline__ uint64_t short_hash(const TableArgs &A, const unsigned long long *d) {
  uint64_t h = A.keys[0];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const uint64_t w = d[i];
    h += A.keys[1 + 2 * i] * (w & 0xffffffffull) + A.keys[2 + 2 * i] * (w >> 32);
  }
  return h;
}

template <int K>
__device__ __forceinline__ bool same_digest(const unsigned long long *a, const unsigned long long *b) {
  bool eq = true;
#pragma unroll
  for (int i = 0; i < K; ++i) eq &= __ldg(a + i) == b[i];
  return eq;
}

// One thread per new entry: claim the first empty slot of its walk, or, at a
// slot holding an equal digest, lower the slot's id to its own if smaller.
template <int K>
__global__ void __launch_bounds__(256) table_insert_kernel(const __grid_constant__ TableArgs A) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long d[K];
#pragma unroll
    for (int j = 0; j < K; ++j) d[j] = __ldg(A.query + i * K + j);
    const unsigned int e = A.base + (unsigned int)i;
    uint64_t s = short_hash<K>(A, d) >> A.shift;
    bool placed = false;
    for (uint64_t probe = 0; probe <= A.mask; ++probe, s = (s + 1) & A.mask) {
      unsigned int cur = __ldcg(A.slots + s);
      if (cur == kEmpty) {
        cur = atomicCAS(A.slots + s, kEmpty, e);
        if (cur == kEmpty) {
          placed = true;
          break;
        }
      }
      if (same_digest<K>(A.rows + (uint64_t)cur * K, d)) {
        atomicMin(A.slots + s, e);
        placed = true;
        break;
      }
    }
    if (!placed) atomicExch(A.status, 1u);
  }
}

// One thread per query: the id in the first slot of its walk that holds an
// equal digest, or kEmpty at the first empty slot.
template <int K>
__global__ void __launch_bounds__(256) table_find_kernel(const __grid_constant__ TableArgs A) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long d[K];
#pragma unroll
    for (int j = 0; j < K; ++j) d[j] = A.query[i * K + j];
    uint64_t s = short_hash<K>(A, d) >> A.shift;
    unsigned int found = kEmpty;
    bool ended = false;
    for (uint64_t probe = 0; probe <= A.mask; ++probe, s = (s + 1) & A.mask) {
      const unsigned int cur = __ldcg(A.slots + s);
      if (cur == kEmpty) {
        ended = true;
        break;
      }
      if (same_digest<K>(A.rows + (uint64_t)cur * K, d)) {
        found = cur;
        ended = true;
        break;
      }
    }
    if (!ended) atomicExch(A.status, 1u);
    A.out[i] = found;
  }
}

const void *insert_kernel(int k) {
  switch (k) {
    case 2: return (const void *)table_insert_kernel<2>;
    case 3: return (const void *)table_insert_kernel<3>;
    case 4: return (const void *)table_insert_kernel<4>;
    case 5: return (const void *)table_insert_kernel<5>;
  }
  return nullptr;
}

const void *find_kernel(int k) {
  switch (k) {
    case 2: return (const void *)table_find_kernel<2>;
    case 3: return (const void *)table_find_kernel<3>;
    case 4: return (const void *)table_find_kernel<4>;
    case 5: return (const void *)table_find_kernel<5>;
  }
  return nullptr;
}

uint64_t short_hash_host(const uint64_t *keys, int k, const uint64_t *d) {
  uint64_t h = keys[0];
  for (int i = 0; i < k; ++i) h += keys[1 + 2 * i] * (d[i] & 0xffffffffull) + keys[2 + 2 * i] * (d[i] >> 32);
  return h;
}

}  // namespace

struct ht_table {
  ht_ctx *ctx = nullptr;
  int k = 0;
  int m = 0;  // log2 of the slot count
  uint64_t max_entries = 0;
  uint64_t entries = 0;
  uint64_t keys[kMaxKeys] = {};
  unsigned long long *rows = nullptr;
  unsigned int *slots = nullptr;
  unsigned int *status = nullptr;
};

namespace {

void table_args(const ht_table *t, TableArgs &A) {
  memset(&A, 0, sizeof A);
  for (int i = 0; i < 2 * t->k + 1; ++i) A.keys[i] = t->keys[i];
  A.rows = t->rows;
  A.slots = t->slots;
  A.status = t->status;
  A.shift = 64 - t->m;
  A.mask = (1ull << t->m) - 1;
}

int launch_table(const ht_table *t, const void *func, TableArgs &A, cudaStream_t s) {
  if (A.count == 0) return HT_OK;
  const uint64_t blocks = std::min<uint64_t>((A.count + 255) / 256, (uint64_t)t->ctx->num_sms * 8);
  void *args[] = {&A};
  cudaError_t e = cudaLaunchKernel(func, dim3((unsigned)blocks), dim3(256), args, 0, s);
  if (e != cudaSuccess) return cuda_error(e, "table kernel launch");
  t->ctx->launches.fetch_add(1);
  return HT_OK;
}

void free_table(ht_table *t) {
  cudaFree(t->rows);
  cudaFree(t->slots);
  cudaFree(t->status);
}

}  // namespace

extern "C" {

int ht_short_hash_keys(uint64_t seed64, int width_bytes, uint64_t *keys_out, size_t n) {
  const KernelSet *ks = kernel_set(width_bytes);
  if (!ks) return set_error(HT_ERR_WIDTH, "unsupported width %d", width_bytes);
  const size_t need = 2 * (size_t)ks->k + 1;
  if (!keys_out || n != need) return set_error(HT_ERR_ARG, "key buffer must hold %zu words (got %zu)", need, n);
  uint64_t st = seed64;
  for (size_t i = 0; i < n; ++i) keys_out[i] = splitmix64_next(&st);
  return HT_OK;
}

int ht_short_hash(const uint64_t *keys, int width_bytes, const uint64_t *digest, uint64_t *out) {
  const KernelSet *ks = kernel_set(width_bytes);
  if (!ks) return set_error(HT_ERR_WIDTH, "unsupported width %d", width_bytes);
  if (!keys || !digest || !out) return set_error(HT_ERR_ARG, "ht_short_hash: NULL argument");
  *out = short_hash_host(keys, ks->k, digest);
  return HT_OK;
}

int ht_table_create(ht_ctx *ctx, uint64_t max_entries, uint64_t seed64, ht_table **out) {
  if (!ctx || !out) return set_error(HT_ERR_ARG, "ht_table_create: NULL argument");
  *out = nullptr;
  if (max_entries == 0 || max_entries > (1ull << 31))
    return set_error(HT_ERR_ARG, "ht_table_create: max_entries must be in 1 .. 2^31");
  ht_table *t = new ht_table;
  t->ctx = ctx;
  t->k = ctx->ks->k;
  t->max_entries = max_entries;
  int m = 1;
  while ((1ull << m) < 2 * max_entries) ++m;  // at most half full
  t->m = m;
  uint64_t st = seed64;
  for (int i = 0; i < 2 * t->k + 1; ++i) t->keys[i] = splitmix64_next(&st);
  cudaError_t e = cudaMalloc((void **)&t->rows, max_entries * t->k * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->slots, (1ull << m) * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(t->slots, 0xff, (1ull << m) * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(t->status, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_table(t);
    delete t;
    return cuda_error(e, "ht_table_create");
  }
  *out = t;
  return HT_OK;
}

int ht_table_destroy(ht_table *t) {
  if (!t) return HT_OK;
  cudaDeviceSynchronize();
  free_table(t);
  delete t;
  return HT_OK;
}

int ht_table_clear(ht_table *t, ht_stream_t stream) {
  if (!t) return set_error(HT_ERR_ARG, "ht_table_clear: NULL table");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(t->slots, 0xff, (1ull << t->m) * sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->status, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_error(e, "ht_table_clear");
  t->entries = 0;
  return HT_OK;
}

uint64_t ht_table_entries(const ht_table *t) { return t ? t->entries : 0; }

int ht_table_slot_bits(const ht_table *t) { return t ? t->m : 0; }

int ht_table_keys(const ht_table *t, uint64_t *keys_out, size_t n) {
  if (!t || !keys_out || n != 2 * (size_t)t->k + 1) return set_error(HT_ERR_ARG, "ht_table_keys: bad arguments");
  for (size_t i = 0; i < n; ++i) keys_out[i] = t->keys[i];
  return HT_OK;
}

int ht_table_insert(ht_table *t, const uint64_t *digests_dev, size_t count, uint32_t *rep_dev,
                    ht_stream_t stream) {
  if (!t || (count && !digests_dev)) return set_error(HT_ERR_ARG, "ht_table_insert: bad arguments");
  if (count > t->max_entries - t->entries)
    return set_error(HT_ERR_BUDGET, "ht_table_insert: %llu entries would exceed the table's %llu",
                     (unsigned long long)(t->entries + count), (unsigned long long)t->max_entries);
  if (count == 0) return HT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *dst = t->rows + t->entries * t->k;
  cudaError_t e = cudaMemcpyAsync(dst, digests_dev, count * t->k * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "ht_table_insert copy");
  TableArgs A;
  table_args(t, A);
  A.query = dst;
  A.count = count;
  A.base = (unsigned int)t->entries;
  int rc = launch_table(t, insert_kernel(t->k), A, s);
  if (rc) return rc;
  t->entries += count;
  if (rep_dev) {
    // after every claim and minimum of the batch: each new entry's walk ends
    // at the slot of its digest, which holds the smallest equal id
    A.out = rep_dev;
    rc = launch_table(t, find_kernel(t->k), A, s);
    if (rc) return rc;
  }
  return HT_OK;
}

int ht_table_find(ht_table *t, const uint64_t *digests_dev, size_t count, uint32_t *found_dev,
                  ht_stream_t stream) {
  if (!t || (count && (!digests_dev || !found_dev))) return set_error(HT_ERR_ARG, "ht_table_find: bad arguments");
  TableArgs A;
  table_args(t, A);
  A.query = reinterpret_cast<const unsigned long long *>(digests_dev);
  A.count = count;
  A.out = found_dev;
  return launch_table(t, find_kernel(t->k), A, (cudaStream_t)stream);
}

int ht_table_status(ht_table *t, ht_stream_t stream) {
  if (!t) return set_error(HT_ERR_ARG, "ht_table_status: NULL table");
  unsigned int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, t->status, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "ht_table_status");
  if (st) return set_error(HT_ERR_BUDGET, "a table walk found no free slot");
  return HT_OK;
}

}  // extern "C"
