// ht_server.cpp -- continuous-batching request loop of libhalftime.
//
// Requests arrive on any thread (ht_server_submit).  A dispatcher thread turns
// the head of the FIFO queue into a batch as soon as a stream slot is free,
// admitting requests while their bytes fit the memory budget.  Pinned-host
// requests that the GPU can address are read in place by the batch kernel
// (on GB300 over the coherent CPU-GPU link: no copy call per request, no
// arena space); others, or all with pinned_mode 1, are staged into a device
// arena carved from that budget.  Each slot
// owns its own context (so its tree scratch never races another slot's), its
// stream and pinned descriptor buffers; a batch is one ht_hash_batch (planner
// + persistent kernel replayed from a graph) followed by a digest copy and an
// event.  A completion thread retires batches as their events fire, copies
// digests to the callers, frees budget and arena space, records latencies and
// wakes the dispatcher and any waiters.  All waits on the host are bounded by
// the caller's timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "halftime.h"
#include "halftime_testing.h"
#include "ht_runtime.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kInFlight = 1, kDone = 2 };

struct Req {
  const void *ptr = nullptr;
  uint64_t len = 0;
  int pinned = 0;
  uint64_t *digest_host = nullptr;
  int64_t t_arrive = 0, t_launch = 0, t_done = 0;
  int state = kQueued;
  int status = HT_OK;
  uint64_t arena_off = 0;
  bool has_arena = false;
  const void *dev_ptr = nullptr;  // pinned request read in place: its device address
};

// First-fit allocator over [0, size) with 256-byte granules.
class Arena {
 public:
  void reset(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(uint64_t bytes, uint64_t *off) {
    bytes = std::max<uint64_t>(256, (bytes + 255) & ~255ull);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = std::max<uint64_t>(256, (bytes + 255) & ~255ull);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<uint64_t, uint64_t> free_;
};

struct Slot {
  bool busy = false;      // owns a batch
  bool launched = false;  // its work is enqueued: safe to poll
  cudaStream_t stream = nullptr;
  ht_ctx *ctx = nullptr;
  cudaEvent_t ev = nullptr;
  const void **h_ptrs = nullptr;
  uint64_t *h_lens = nullptr;
  uint64_t *h_digests = nullptr;
  const void **d_ptrs = nullptr;
  uint64_t *d_lens = nullptr;
  uint64_t *d_digests = nullptr;
  // device views of h_ptrs, h_lens and h_digests when the GPU can address
  // pinned host memory (and requests are not forced through staging): the
  // planner then reads the descriptors and the batch kernel writes the
  // digests in place, with no copy in either direction (else null)
  const void **m_ptrs = nullptr;
  uint64_t *m_lens = nullptr;
  uint64_t *m_digests = nullptr;
  std::vector<uint64_t> tickets;
  uint64_t bytes = 0;
  int64_t fake_deadline = 0;
  bool fake_fail = false;
  int launch_status = HT_OK;
};

}  // namespace

struct ht_server {
  // configuration
  int width = 0, k = 0;
  bool fake = false;
  uint64_t fake_delay_us = 0;
  int64_t fake_fail_batch = -1;
  uint64_t budget = 0;
  ht_server_opts opts = {};
  // device resources
  uint8_t *arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  // state
  std::mutex mu;
  std::condition_variable cv_dispatch, cv_complete, cv_done;
  std::deque<Req> reqs;  // index = ticket
  std::deque<uint64_t> queue;
  uint64_t in_use = 0;
  uint64_t batches = 0, rejected = 0, completed = 0, bytes_completed = 0;
  std::vector<double> lat_us;
  int64_t first_arrive = 0, last_done = 0;
  bool stop = false;
  std::thread dispatcher, completer;
};

namespace {

// Batches of at most this many requests run as single-string launches, one
// per request, instead of the batch graph (four planner launches and the
// batch kernels).  Measured on GB300 (width 32, C5 request mix, eight
// batches in flight, p50 at 10 / 30 / 50 / 70 / 90 % load): all batches
// through the graph but lone requests 41-53 / 112 / 154-163 / 263-269 /
// 653-703 us; up to 4 singles 34 / 78 / 121 / 259-281 / 652-788; up to 8
// singles 35 / 90 / 113 / 186-195 / 512-533 (p99 at 90 %: 0.96-1.16 ms
// against 1.21-1.38); up to 16 or 32 singles slower again from 30 % load.
constexpr size_t kSingleLaunches = 8;

// Enqueues a formed batch: staging copies of pinned requests that the GPU
// cannot read in place, then one single-string launch (a lone request) or the
// batch graph, with descriptor and digest copies only where the GPU cannot
// address the slot's pinned buffers, then the slot's completion event.
int launch_real(ht_server *S, Slot &sl, const std::vector<Req *> &batch) {
  const size_t n = batch.size();
  for (size_t i = 0; i < n; ++i) {
    Req *r = batch[i];
    if (r->dev_ptr) {
      sl.h_ptrs[i] = r->dev_ptr;  // read in place over the CPU-GPU link
    } else if (r->pinned && r->len) {
      uint8_t *dst = S->arena_base + r->arena_off;
      cudaError_t e = cudaMemcpyAsync(dst, r->ptr, r->len, cudaMemcpyHostToDevice, sl.stream);
      if (e != cudaSuccess) return ht::cuda_error(e, "request staging copy");
      sl.h_ptrs[i] = dst;
    } else {
      sl.h_ptrs[i] = r->ptr;
    }
    sl.h_lens[i] = r->len;
  }
  cudaError_t e = cudaSuccess;
  if (n <= kSingleLaunches) {
    // a few requests (common at low load): one single-string launch each
    // instead of the batch graph's planner and batch kernels
    uint64_t *dig = sl.m_digests ? sl.m_digests : sl.d_digests;
    for (size_t i = 0; i < n; ++i) {
      int rc = ht_hash(sl.ctx, sl.h_ptrs[i], sl.h_lens[i], dig + i * S->k, sl.stream);
      if (rc) return rc;
    }
    if (!sl.m_digests)
      e = cudaMemcpyAsync(sl.h_digests, sl.d_digests, n * S->k * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                          sl.stream);
  } else if (sl.m_ptrs) {
    // descriptors read and digests written in place: the batch graph is the
    // only work of the batch (the stores above precede the launch)
    std::atomic_thread_fence(std::memory_order_release);
    int rc = ht_hash_batch(sl.ctx, sl.m_ptrs, sl.m_lens, n, sl.m_digests, sl.stream);
    if (rc) return rc;
  } else {
    e = cudaMemcpyAsync(sl.d_ptrs, sl.h_ptrs, n * sizeof(void *), cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.d_lens, sl.h_lens, n * sizeof(uint64_t), cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return ht::cuda_error(e, "batch descriptor copy");
    int rc = ht_hash_batch(sl.ctx, sl.d_ptrs, sl.d_lens, n, sl.d_digests, sl.stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(sl.h_digests, sl.d_digests, n * S->k * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                        sl.stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
  if (e != cudaSuccess) return ht::cuda_error(e, "batch digest copy");
  return HT_OK;
}

// 1 = finished, 0 = running, < 0 = error.
int poll_slot(ht_server *S, Slot &sl) {
  if (sl.launch_status != HT_OK) return sl.launch_status;
  if (S->fake) {
    if (now_ns() < sl.fake_deadline) return 0;
    return sl.fake_fail ? ht::set_error(HT_ERR_CUDA, "injected batch failure") : 1;
  }
  cudaError_t e = cudaEventQuery(sl.ev);
  if (e == cudaErrorNotReady) return 0;
  if (e != cudaSuccess) return ht::cuda_error(e, "batch event");
  return 1;
}

// The device address of a pinned request that the batch kernel can read in
// place (pinned host memory the GPU addresses directly), or null: then the
// request is staged through the arena.
const void *in_place_address(const ht_server *S, const void *ptr, uint64_t len, int pinned) {
  if (!pinned || !len || S->fake || S->opts.pinned_mode != 0) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // (clears the error: not a device-visible allocation)
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}

void release_req(ht_server *S, Req &r) {
  if (r.has_arena) {
    S->arena.release(r.arena_off, r.len);
    r.has_arena = false;
  }
  S->in_use -= r.len;
}

void dispatcher_main(ht_server *S) {
  if (!S->fake && !S->slots.empty()) cudaSetDevice(S->slots[0].ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    Slot *free_slot = nullptr;
    S->cv_dispatch.wait(lk, [&] {
      if (S->stop) return true;
      if (S->queue.empty()) return false;
      for (auto &sl : S->slots)
        if (!sl.busy) return true;
      return false;
    });
    if (S->stop) break;
    // optional batching window: wait a little for batch-mates
    if (S->opts.max_wait_us && S->queue.size() < S->opts.max_batch) {
      const int64_t oldest = S->reqs[S->queue.front()].t_arrive;
      const int64_t until = oldest + (int64_t)S->opts.max_wait_us * 1000;
      while (!S->stop && S->queue.size() < S->opts.max_batch && now_ns() < until)
        S->cv_dispatch.wait_for(lk, std::chrono::nanoseconds(std::max<int64_t>(until - now_ns(), 1000)));
      if (S->stop) break;
      if (S->queue.empty()) continue;
    }
    for (auto &sl : S->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) continue;
    std::vector<Req *> batch;
    std::vector<uint64_t> tickets;
    uint64_t bytes = 0;
    while (!S->queue.empty() && batch.size() < S->opts.max_batch) {
      Req &r = S->reqs[S->queue.front()];
      if (S->in_use + r.len > S->budget) break;
      if (r.pinned && r.len && !r.dev_ptr) {
        if (!S->arena.alloc(r.len, &r.arena_off)) break;
        r.has_arena = true;
      }
      S->in_use += r.len;
      bytes += r.len;
      r.state = kInFlight;
      batch.push_back(&r);
      tickets.push_back(S->queue.front());
      S->queue.pop_front();
    }
    if (batch.empty()) {
      // the head does not fit until in-flight work retires
      S->cv_dispatch.wait_for(lk, std::chrono::milliseconds(1));
      continue;
    }
    Slot &sl = *free_slot;
    sl.busy = true;
    sl.tickets = tickets;
    sl.bytes = bytes;
    const int64_t t = now_ns();
    for (Req *r : batch) r->t_launch = t;
    const uint64_t batch_no = S->batches++;
    lk.unlock();
    int rc = HT_OK;
    if (S->fake) {
      sl.fake_deadline = now_ns() + (int64_t)S->fake_delay_us * 1000;
      sl.fake_fail = ((int64_t)batch_no == S->fake_fail_batch);
      for (size_t i = 0; i < batch.size(); ++i)
        memset(sl.h_digests + i * S->k, 0, S->k * sizeof(uint64_t));
    } else {
      rc = launch_real(S, sl, batch);
    }
    lk.lock();
    sl.launch_status = rc;
    sl.launched = true;
    S->cv_complete.notify_all();
  }
}

// Retires batches.  Event queries run without the server lock (a busy,
// launched slot is only touched by this thread until it is retired), so
// submitters and the dispatcher are not held up while the GPU works.
void completer_main(ht_server *S) {
  if (!S->fake && !S->slots.empty()) cudaSetDevice(S->slots[0].ctx->device);
  std::vector<size_t> watch, done;
  std::vector<int> codes;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      watch.clear();
      bool any_busy = false;
      for (size_t i = 0; i < S->slots.size(); ++i)
        if (S->slots[i].busy) {
          any_busy = true;
          if (S->slots[i].launched) watch.push_back(i);
        }
      if (S->stop && !any_busy) return;
      if (watch.empty()) {
        S->cv_complete.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    done.clear();
    codes.clear();
    for (size_t i : watch) {
      const int rc = poll_slot(S, S->slots[i]);
      if (rc != 0) {
        done.push_back(i);
        codes.push_back(rc);
      }
    }
    if (done.empty()) {
      std::this_thread::yield();
      continue;
    }
    const int64_t t = now_ns();
    std::lock_guard<std::mutex> g(S->mu);
    for (size_t d = 0; d < done.size(); ++d) {
      Slot &sl = S->slots[done[d]];
      const int rc = codes[d];
      for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Req &r = S->reqs[sl.tickets[i]];
        if (rc == 1 && r.digest_host) memcpy(r.digest_host, sl.h_digests + i * S->k, S->k * sizeof(uint64_t));
        r.status = rc == 1 ? HT_OK : rc;
        r.state = kDone;
        r.t_done = t;
        release_req(S, r);
        if (rc == 1) {
          S->completed++;
          S->bytes_completed += r.len;
          S->lat_us.push_back((r.t_done - r.t_arrive) / 1000.0);
          if (!S->first_arrive || r.t_arrive < S->first_arrive) S->first_arrive = r.t_arrive;
          S->last_done = std::max(S->last_done, t);
        }
      }
      sl.tickets.clear();
      sl.busy = false;
      sl.launched = false;
      sl.launch_status = HT_OK;
    }
    S->cv_dispatch.notify_all();
    S->cv_done.notify_all();
  }
}

int make_server(ht_server *S, ht_ctx *ctx, uint64_t budget, const ht_server_opts *opts) {
  S->budget = budget;
  ht_server_opts o;
  // eight batches in flight: on GB300 with width 32, requests of 256 B ..
  // 64 MiB at 90 % of the burst peak, p50 / p99 0.69 / 1.32 ms against
  // 0.81-0.91 / 1.74-1.99 ms with four (three runs each); 16 were no better
  o.n_streams = 8;
  o.max_batch = 4096;
  o.max_queue = 1u << 20;
  o.max_wait_us = 0;
  o.pinned_mode = 0;
  if (opts) {
    if (opts->n_streams > 0) o.n_streams = opts->n_streams;
    if (opts->max_batch > 0) o.max_batch = opts->max_batch;
    if (opts->max_queue > 0) o.max_queue = opts->max_queue;
    o.max_wait_us = opts->max_wait_us;
    o.pinned_mode = opts->pinned_mode;
  }
  S->opts = o;
  S->slots.resize((size_t)o.n_streams);
  if (S->fake) {
    S->arena.reset(budget);
    for (auto &sl : S->slots) sl.h_digests = new uint64_t[o.max_batch * S->k];
    return HT_OK;
  }
  cudaError_t e = cudaMalloc((void **)&S->arena_base, std::max<uint64_t>(budget, 256));
  if (e != cudaSuccess) return ht::cuda_error(e, "server arena");
  S->arena.reset(budget);
  for (auto &sl : S->slots) {
    int rc = ht_ctx_create(ctx->width, ctx->h_seeds.data(), ctx->h_seeds.size(), nullptr, &sl.ctx);
    if (rc) return rc;
    rc = ht_ctx_reserve(sl.ctx, budget, o.max_batch);
    if (rc) return rc;
    // every length bucket's launch shape (a lone request is a single-string
    // launch) and the batch shape
    for (int b = 0; b < 65; ++b) sl.ctx->shapes[b] = ctx->shapes[b];
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_ptrs, o.max_batch * sizeof(void *));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_lens, o.max_batch * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_digests, o.max_batch * S->k * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_ptrs, o.max_batch * sizeof(void *));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_lens, o.max_batch * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_digests, o.max_batch * S->k * sizeof(uint64_t));
    if (e != cudaSuccess) return ht::cuda_error(e, "server slot");
    if (o.pinned_mode == 0) {
      // the same buffers as the GPU sees them, if it can address them
      void *mp = nullptr, *ml = nullptr, *md = nullptr;
      if (cudaHostGetDevicePointer(&mp, (void *)sl.h_ptrs, 0) == cudaSuccess &&
          cudaHostGetDevicePointer(&ml, sl.h_lens, 0) == cudaSuccess &&
          cudaHostGetDevicePointer(&md, sl.h_digests, 0) == cudaSuccess) {
        sl.m_ptrs = static_cast<const void **>(mp);
        sl.m_lens = static_cast<uint64_t *>(ml);
        sl.m_digests = static_cast<uint64_t *>(md);
      } else {
        cudaGetLastError();  // (not mapped: the descriptors are copied)
      }
    }
  }
  return HT_OK;
}

void free_server(ht_server *S) {
  if (S->fake) {
    for (auto &sl : S->slots) delete[] sl.h_digests;
  } else {
    for (auto &sl : S->slots) {
      if (sl.stream) cudaStreamSynchronize(sl.stream);
      if (sl.ctx) ht_ctx_destroy(sl.ctx);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.ev) cudaEventDestroy(sl.ev);
      cudaFreeHost(sl.h_ptrs);
      cudaFreeHost(sl.h_lens);
      cudaFreeHost(sl.h_digests);
      cudaFree(sl.d_ptrs);
      cudaFree(sl.d_lens);
      cudaFree(sl.d_digests);
    }
    cudaFree(S->arena_base);
  }
  delete S;
}

void start_threads(ht_server *S) {
  S->dispatcher = std::thread(dispatcher_main, S);
  S->completer = std::thread(completer_main, S);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int ht_server_create(ht_ctx *ctx, uint64_t budget_bytes, const ht_server_opts *opts, ht_server **out) {
  if (!ctx || !out || budget_bytes == 0) return ht::set_error(HT_ERR_ARG, "ht_server_create: bad arguments");
  *out = nullptr;
  ht_server *S = new ht_server();
  S->width = ctx->width;
  S->k = ctx->ks->k;
  int rc = make_server(S, ctx, budget_bytes, opts);
  if (rc) {
    free_server(S);
    return rc;
  }
  start_threads(S);
  *out = S;
  return HT_OK;
}

int ht_server_create_fake(int width, uint64_t budget_bytes, const ht_server_opts *opts,
                          uint64_t batch_delay_us, int64_t fail_batch, ht_server **out) {
  if (width != 16 && width != 24 && width != 32 && width != 40)
    return ht::set_error(HT_ERR_WIDTH, "unsupported width %d", width);
  if (!out || budget_bytes == 0) return ht::set_error(HT_ERR_ARG, "ht_server_create_fake: bad arguments");
  ht_server *S = new ht_server();
  S->width = width;
  S->k = width / 8;
  S->fake = true;
  S->fake_delay_us = batch_delay_us;
  S->fake_fail_batch = fail_batch;
  int rc = make_server(S, nullptr, budget_bytes, opts);
  if (rc) {
    free_server(S);
    return rc;
  }
  start_threads(S);
  *out = S;
  return HT_OK;
}

int ht_server_submit(ht_server *S, const void *ptr, uint64_t len, int pinned, uint64_t *digest_host,
                     uint64_t *ticket) {
  if (!S || !ticket || !digest_host || (len && !ptr))
    return ht::set_error(HT_ERR_ARG, "ht_server_submit: bad arguments");
  if (len > S->budget) {
    std::lock_guard<std::mutex> g(S->mu);
    S->rejected++;
    return ht::set_error(HT_ERR_BUDGET, "request of %llu bytes exceeds the budget of %llu",
                         (unsigned long long)len, (unsigned long long)S->budget);
  }
  const void *dev = in_place_address(S, ptr, len, pinned);
  std::lock_guard<std::mutex> g(S->mu);
  if (S->queue.size() >= S->opts.max_queue) {
    S->rejected++;
    return ht::set_error(HT_ERR_BUSY, "server queue full");
  }
  Req r;
  r.ptr = ptr;
  r.len = len;
  r.pinned = pinned ? 1 : 0;
  r.dev_ptr = dev;
  r.digest_host = digest_host;
  r.t_arrive = now_ns();
  S->reqs.push_back(r);
  *ticket = S->reqs.size() - 1;
  S->queue.push_back(*ticket);
  S->cv_dispatch.notify_one();
  return HT_OK;
}

int ht_server_poll(ht_server *S, uint64_t ticket, int *done) {
  if (!S || !done) return ht::set_error(HT_ERR_ARG, "ht_server_poll: bad arguments");
  std::lock_guard<std::mutex> g(S->mu);
  if (ticket >= S->reqs.size()) return ht::set_error(HT_ERR_ARG, "unknown ticket");
  const Req &r = S->reqs[ticket];
  *done = r.state == kDone;
  return r.state == kDone ? r.status : HT_OK;
}

int ht_server_wait(ht_server *S, uint64_t ticket, uint64_t timeout_us) {
  if (!S) return ht::set_error(HT_ERR_ARG, "ht_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket >= S->reqs.size()) return ht::set_error(HT_ERR_ARG, "unknown ticket");
  const bool ok = S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                      [&] { return S->reqs[ticket].state == kDone; });
  if (!ok) return ht::set_error(HT_ERR_TIMEOUT, "request %llu not done after %llu us",
                                (unsigned long long)ticket, (unsigned long long)timeout_us);
  const int st = S->reqs[ticket].status;
  if (st != HT_OK) return ht::set_error(st, "request %llu failed (%d)", (unsigned long long)ticket, st);
  return HT_OK;
}

int ht_server_drain(ht_server *S, uint64_t timeout_us) {
  if (!S) return ht::set_error(HT_ERR_ARG, "ht_server_drain: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
    if (!S->queue.empty()) return false;
    for (auto &sl : S->slots)
      if (sl.busy) return false;
    return true;
  });
  return ok ? HT_OK : ht::set_error(HT_ERR_TIMEOUT, "server not drained after %llu us",
                                    (unsigned long long)timeout_us);
}

int ht_server_replay(ht_server *S, const void *const *ptrs, const uint64_t *lens, const int *pinned,
                     const double *arrival_us, size_t n, uint64_t *digests_host, uint64_t timeout_us,
                     double *late_us) {
  if (!S || (n && (!ptrs || !lens || !arrival_us || !digests_host)))
    return ht::set_error(HT_ERR_ARG, "ht_server_replay: bad arguments");
  for (size_t i = 0; i < n; ++i)
    if (lens[i] > S->budget)
      return ht::set_error(HT_ERR_BUDGET, "request %zu of %llu bytes exceeds the budget", i,
                           (unsigned long long)lens[i]);
  std::vector<const void *> dev(n, nullptr);  // in-place addresses, resolved before the clock starts
  for (size_t i = 0; i < n; ++i) dev[i] = in_place_address(S, ptrs[i], lens[i], pinned ? pinned[i] : 0);
  const size_t first = S->reqs.size();  // tickets are consecutive from here
  const int64_t t0 = now_ns();
  double worst = 0.0;
  size_t i = 0;
  while (i < n) {
    const int64_t due = t0 + (int64_t)(arrival_us[i] * 1000.0);
    int64_t now = now_ns();
    while (now < due) now = now_ns();
    // every request due by now goes in under one lock acquisition
    std::lock_guard<std::mutex> g(S->mu);
    size_t j = i;
    while (j < n && t0 + (int64_t)(arrival_us[j] * 1000.0) <= now && S->queue.size() < S->opts.max_queue) {
      Req r;
      r.ptr = ptrs[j];
      r.len = lens[j];
      r.pinned = pinned ? (pinned[j] ? 1 : 0) : 0;
      r.dev_ptr = dev[j];
      r.digest_host = digests_host + j * (size_t)S->k;
      r.t_arrive = t0 + (int64_t)(arrival_us[j] * 1000.0);  // scheduled arrival
      S->reqs.push_back(r);
      S->queue.push_back(S->reqs.size() - 1);
      worst = std::max(worst, (now - r.t_arrive) / 1000.0);
      ++j;
    }
    if (j > i) S->cv_dispatch.notify_one();
    i = j;
  }
  if (late_us) *late_us = worst;
  int first_err = HT_OK;
  for (size_t t = 0; t < n; ++t) {
    const int rc = ht_server_wait(S, first + t, timeout_us);
    if (rc != HT_OK && first_err == HT_OK) first_err = rc;
  }
  return first_err;
}

int ht_server_cancel(ht_server *S, uint64_t ticket) {
  if (!S) return ht::set_error(HT_ERR_ARG, "ht_server_cancel: NULL server");
  std::lock_guard<std::mutex> g(S->mu);
  if (ticket >= S->reqs.size()) return ht::set_error(HT_ERR_ARG, "unknown ticket");
  Req &r = S->reqs[ticket];
  if (r.state != kQueued) return ht::set_error(HT_ERR_BUSY, "request already launched");
  auto it = std::find(S->queue.begin(), S->queue.end(), ticket);
  if (it != S->queue.end()) S->queue.erase(it);
  r.state = kDone;
  r.status = HT_ERR_ARG;
  r.t_done = now_ns();
  S->cv_done.notify_all();
  return HT_OK;
}

int ht_server_stats(ht_server *S, ht_server_stats_t *out, int reset) {
  if (!S || !out) return ht::set_error(HT_ERR_ARG, "ht_server_stats: bad arguments");
  std::lock_guard<std::mutex> g(S->mu);
  out->submitted = S->reqs.size();
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->batches = S->batches;
  out->bytes_completed = S->bytes_completed;
  out->p50_us = percentile(S->lat_us, 0.50);
  out->p99_us = percentile(S->lat_us, 0.99);
  double sum = 0, mx = 0;
  for (double v : S->lat_us) {
    sum += v;
    mx = std::max(mx, v);
  }
  out->mean_us = S->lat_us.empty() ? 0.0 : sum / (double)S->lat_us.size();
  out->max_us = mx;
  out->wall_s = (S->last_done > S->first_arrive) ? (S->last_done - S->first_arrive) * 1e-9 : 0.0;
  if (reset) {
    S->lat_us.clear();
    S->completed = 0;
    S->bytes_completed = 0;
    S->first_arrive = 0;
    S->last_done = 0;
  }
  return HT_OK;
}

size_t ht_server_latencies(ht_server *S, double *out_us, size_t n) {
  if (!S || !out_us) return 0;
  std::lock_guard<std::mutex> g(S->mu);
  const size_t m = std::min(n, S->lat_us.size());
  std::copy(S->lat_us.begin(), S->lat_us.begin() + (ptrdiff_t)m, out_us);
  return m;
}

int ht_server_destroy(ht_server *S) {
  if (!S) return HT_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_dispatch.notify_all();
  S->cv_complete.notify_all();
  if (S->dispatcher.joinable()) S->dispatcher.join();
  if (S->completer.joinable()) S->completer.join();
  free_server(S);
  return HT_OK;
}

}  // extern "C"
