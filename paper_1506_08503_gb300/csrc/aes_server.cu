// aes_server.cu -- request server with continuous batching over the batched T-table launch.
//
// The paper's point (Sections III-IV) is throughput on many small messages by processing
// them together; a server adds the time dimension: requests arrive one by one.  The server's
// thread keeps a FIFO of submitted requests and, whenever one of its CUDA streams is idle,
// admits as many queued requests as the in-flight limit, the batch size and the free staging
// memory allow, and starts them as ONE batched launch on that stream:
//   host payloads that the kernel can reach itself (a device with direct access to host
//   memory, 16-byte aligned buffers) are read and written in place; other host-sourced
//   payloads are copied into the staging arena (or straight into a device destination), the
//   batch graph runs the cipher, and other host destinations are copied back; an event at
//   the end of the stream marks the batch done, and the server's thread, which polls the
//   events of its batches in flight, then marks the batch's requests complete, frees their
//   staging and wakes any waiting poll.
// Requests arriving while batches run are admitted into the next free stream's batch, so the
// device works on several batches at once and nobody waits for a full drain.
//
// Threads: the worker admits (under the server mutex) and retires; each stream slot has an issuer
// thread that builds the admitted batch's descriptors and launches it, so the host work of
// several batches (linear in their request counts) proceeds in parallel.  A bulk submission
// reserves all its tickets at once and writes them in chunks, so admission starts before the
// whole submission is written.
//
// Staging memory is one cudaMalloc'd arena (the HBM budget) managed by a first-fit free list
// with coalescing; a request is admitted only when its staging fits (head-of-line order is
// kept, so large requests are not starved by small ones).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "aes_internal.cuh"
#include "aesgb_testing.h"

namespace {

using namespace aesgb;
using Clock = std::chrono::steady_clock;
constexpr size_t kLatencyWindow = size_t(1) << 22;  // latencies kept for p50/p99

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// First-fit allocator over [0, size) with 256-byte granularity and coalescing frees.
class Arena {
 public:
  explicit Arena(size_t size = 0) { reset(size); }
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

// One request slot of the ring.  Ticket t lives in ring[t & mask] from submission until a
// poll releases it.  `ticket` (0 = free) is stored last, with release order, once the request
// is in place; `state` moves PENDING -> DONE or FAILED once.  Both are atomic because the
// thread that owns a reserved or in-flight ticket range writes them without the server mutex.
struct Req {
  aes_request r{};
  double t_submit = 0;
  size_t stage_off = 0, stage_bytes = 0;
  bool staged = false;
  std::atomic<int> state{AES_REQ_PENDING};
  std::atomic<uint64_t> ticket{0};
};

struct StreamSlot {
  cudaStream_t stream = nullptr;
  aes_batch* batch = nullptr;
  bool busy = false;         // admitted and not yet retired
  bool pending = false;      // admitted, waiting for this slot's issuer thread
  bool inject_fail = false;  // fault injection: the issuer fails this batch
  uint64_t first = 0, last = 0;  // the batch is the ticket range [first, last)
  cudaEvent_t done_ev = nullptr;  // recorded after the batch's last operation on the stream
  std::atomic<bool> awaiting{false};  // issued: the worker polls done_ev and retires the batch
  StreamSlot() = default;
  StreamSlot(const StreamSlot&) = delete;
  StreamSlot& operator=(const StreamSlot&) = delete;
  std::vector<double> lat;   // retirement scratch (max_batch entries)
  std::vector<std::pair<size_t, size_t>> frees;
};


}  // namespace

struct aes_server {
  aes_server_cfg cfg{};
  aes_keypool* pool = nullptr;
  int device = -1;
  uint8_t* arena_base = nullptr;
  Arena arena;
  bool host_direct = false;  // kernels may load and store host memory (see DeviceInfo)
  std::deque<StreamSlot> slots;  // a deque: the slots hold atomics and are never moved

  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_issue;
  std::unique_ptr<Req[]> ring;  // power-of-two size >= queue_capacity
  uint64_t ring_size = 0;
  uint64_t mask = 0;
  uint64_t next_ticket = 1;    // next ticket to hand out (tickets below it are reserved)
  uint64_t filled = 1;         // first ticket whose request is not yet in the ring
  uint64_t oldest = 1;         // first ticket not yet released by a poll
  uint64_t admit = 1;          // first ticket not admitted yet: the queue is [admit, filled)
  uint64_t inflight = 0;
  bool stop = false;
  bool stop_issuers = false;
  std::thread worker;
  std::vector<std::thread> issuers;  // one per stream slot

  // statistics
  // latencies of the most recent completions (a ring of kLatencyWindow entries, so a server
  // that runs for days keeps bounded memory); lat_n counts all recorded since the last reset
  std::vector<double> lat_us;
  uint64_t lat_n = 0;
  uint64_t submitted = 0, completed = 0, failed = 0, launches = 0, launched_reqs = 0, bytes_done = 0;
  double t_first = 0, t_last = 0, t_first_launch = 0;

  Req& at(uint64_t t) { return ring[t & mask]; }
};

namespace {

// A buffer the kernel reads or writes itself: device memory, or host memory on a device that
// accesses host memory directly (16-byte aligned, for 128-bit accesses).  Other host buffers
// are copied through the staging arena.
bool src_direct(const aes_server* s, const aes_request& r) {
  return r.src_on_device || (s->host_direct && (reinterpret_cast<uintptr_t>(r.src) & 15u) == 0);
}
bool dst_direct(const aes_server* s, const aes_request& r) {
  return r.dst_on_device || (s->host_direct && (reinterpret_cast<uintptr_t>(r.dst) & 15u) == 0);
}
// Staging holds the output for a destination that is not direct, and the input for a source
// that is not direct when the destination is not device memory (a device destination takes
// the copied input and is enciphered in place).
bool needs_staging(const aes_server* s, const aes_request& r) {
  return !dst_direct(s, r) || (!src_direct(s, r) && !r.dst_on_device);
}

// Finishes a slot's batch: every request's state becomes `state` (DONE or FAILED), then the
// counters, latencies and staging frees are applied under the mutex in one step.  The slot's
// ticket range belongs to the batch until its states are stored, so the per-request pass
// needs no lock; a request is not touched after its state store (a poll may then release and
// reuse its slot).  Waiters are woken after the locked step, so no wake-up is lost.  Called
// WITHOUT mu held.
void retire(aes_server* s, StreamSlot& sl, double t, int state) {
  sl.lat.clear();
  sl.frees.clear();
  uint64_t bytes = 0;
  const uint64_t n = sl.last - sl.first;
  for (uint64_t tk = sl.first; tk < sl.last; ++tk) {
    Req& q = s->at(tk);
    if (q.staged) sl.frees.emplace_back(q.stage_off, q.stage_bytes);
    q.staged = false;
    bytes += q.r.length;
    if (state == AES_REQ_DONE) sl.lat.push_back((t - q.t_submit) * 1e6);
    q.state.store(state, std::memory_order_release);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const auto& f : sl.frees) s->arena.release(f.first, f.second);
    s->inflight -= n;
    if (state == AES_REQ_DONE) {
      s->completed += n;
      s->bytes_done += bytes;
      for (double v : sl.lat) {
        if (s->lat_us.size() < kLatencyWindow) s->lat_us.push_back(v);
        else s->lat_us[s->lat_n % kLatencyWindow] = v;
        ++s->lat_n;
      }
      if (t > s->t_last) s->t_last = t;
    } else {
      s->failed += n;
    }
    sl.busy = false;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_one();
}

aes_status issue_batched(aes_server* s, StreamSlot& sl, cudaStream_t st, size_t nenc, size_t ndec);

// Issues the tickets [sl.first, sl.last) on slot i (mu NOT held; the batch owns its ring
// slots until the worker sees its done event and retires them).
aes_status issue(aes_server* s, int i) {
  StreamSlot& sl = s->slots[i];
  cudaStream_t st = sl.stream;
  cudaError_t e;
  if (sl.inject_fail) return set_error(AES_ECUDA, "injected launch failure (fail_every = %u)", s->cfg.fail_every);
  // pass 1: host payloads go to the device, and the batch is counted per direction
  size_t nenc = 0, ndec = 0;
  uint64_t nblocks = 0;
  for (uint64_t tk = sl.first; tk < sl.last; ++tk) {
    const Req& q = s->at(tk);
    const aes_request& r = q.r;
    if (!src_direct(s, r)) {
      void* to = r.dst_on_device ? r.dst : static_cast<void*>(s->arena_base + q.stage_off);
      if ((e = cudaMemcpyAsync(to, r.src, r.length, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_error(e, "H2D");
    }
    (r.dir == AES_ENCRYPT ? nenc : ndec)++;
    nblocks += r.length / 16;
  }
  // pass 2 (inside the batch launch): descriptors written straight into the pinned staging.
  // A device destination is the output; a host destination is served from the staging slot,
  // which also holds the input when the source was on the host.
  const uint64_t nreq = sl.last - sl.first;
  if (nreq <= uint64_t(kSmallBatchMax) && nblocks <= kSmallCallBlocks) {
    // a small batch (the common case at low request rates): its descriptors travel as kernel
    // parameters and its tables come from global memory, so it costs one kernel launch: no
    // descriptor upload, no copy-stream event, no graph update, no shared-memory table fill
    SmallBatch b{};
    uint64_t pos = 0;
    for (uint64_t tk = sl.first; tk < sl.last; ++tk) {
      const Req& q = s->at(tk);
      const aes_request& r = q.r;
      const uint64_t stage = reinterpret_cast<uint64_t>(s->arena_base + q.stage_off);
      const uint64_t out_addr = dst_direct(s, r) ? reinterpret_cast<uint64_t>(r.dst) : stage;
      const uint64_t in_addr = src_direct(s, r) ? reinterpret_cast<uint64_t>(r.src)
                               : r.dst_on_device ? reinterpret_cast<uint64_t>(r.dst) : stage;
      SmallMsg& m = b.m[b.n];
      m = SmallMsg{in_addr, out_addr, uint32_t(r.length / 16), r.key_idx, r.dir, 0u};
      b.start[b.n++] = pos;
      pos += r.length / 16;
    }
    b.start[b.n] = pos;
    aes_status rc = launch_small_batch(b, s->pool->entries, st);
    if (rc != AES_OK) return rc;
  } else {
    aes_status rc = issue_batched(s, sl, st, nenc, ndec);
    if (rc != AES_OK) return rc;
  }
  for (uint64_t tk = sl.first; tk < sl.last; ++tk) {
    const Req& q = s->at(tk);
    if (!dst_direct(s, q.r))
      if ((e = cudaMemcpyAsync(q.r.dst, s->arena_base + q.stage_off, q.r.length, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e, "D2H");
  }
  if ((e = cudaEventRecord(sl.done_ev, st)) != cudaSuccess) return cuda_error(e, "cudaEventRecord(batch done)");
  return AES_OK;
}

// The batched launch of a larger batch: descriptors into the pinned staging, then the cached
// graph (batch_launch_descs).
aes_status issue_batched(aes_server* s, StreamSlot& sl, cudaStream_t st, size_t nenc, size_t ndec) {
  auto fill = [&](BatchMsg* em, BatchMsg* dm, uint4*, uint4*) {
    size_t ie = 0, id = 0;
    for (uint64_t tk = sl.first; tk < sl.last; ++tk) {
      const Req& q = s->at(tk);
      const aes_request& r = q.r;
      const uint64_t stage = reinterpret_cast<uint64_t>(s->arena_base + q.stage_off);
      const uint64_t out_addr = dst_direct(s, r) ? reinterpret_cast<uint64_t>(r.dst) : stage;
      const uint64_t in_addr = src_direct(s, r) ? reinterpret_cast<uint64_t>(r.src)
                               : r.dst_on_device ? reinterpret_cast<uint64_t>(r.dst) : stage;
      const BatchMsg d{r.key_idx, 0u, in_addr / 16, out_addr / 16, r.length / 16};
      if (r.dir == AES_ENCRYPT) em[ie++] = d;
      else dm[id++] = d;
    }
  };
  return batch_launch_descs(sl.batch, nenc, ndec, fill, false, 0, 0, st);
}

// A slot's batch has been issued: the worker polls its done event from now on.  Called with
// mu held, so the worker, which checks the flags under mu before it sleeps, cannot miss it.
void mark_issued(aes_server* s, StreamSlot& sl) {
  sl.awaiting.store(true, std::memory_order_release);
  s->cv_work.notify_one();
}

bool any_awaiting(const aes_server* s) {
  for (const StreamSlot& sl : s->slots)
    if (sl.awaiting.load(std::memory_order_acquire)) return true;
  return false;
}

// Retires every issued batch whose done event has fired (mu NOT held: the event queries do
// not block the submitters and pollers).  Returns whether a batch is still in flight.
bool poll_completions(aes_server* s) {
  bool in_flight = false;
  for (StreamSlot& sl : s->slots) {
    if (!sl.awaiting.load(std::memory_order_acquire)) continue;
    const cudaError_t q = cudaEventQuery(sl.done_ev);
    if (q == cudaErrorNotReady) {
      in_flight = true;
      continue;
    }
    sl.awaiting.store(false, std::memory_order_relaxed);
    retire(s, sl, now_s(), q == cudaSuccess ? AES_REQ_DONE : AES_REQ_FAILED);
  }
  return in_flight;
}

// One thread per stream slot builds and launches the slot's batches, so that the descriptor
// work of several batches (linear in their request counts) runs in parallel while the worker
// keeps admitting.
void issuer_main(aes_server* s, int i) {
  cudaSetDevice(s->device);
  StreamSlot& sl = s->slots[i];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_issue.wait(lk, [&] { return sl.pending || s->stop_issuers; });
    if (!sl.pending) break;
    sl.pending = false;
    lk.unlock();
    const aes_status rc = issue(s, i);
    if (rc != AES_OK) {
      cudaStreamSynchronize(sl.stream);  // copies queued before the failure may still read the staging
      retire(s, sl, now_s(), AES_REQ_FAILED);
    }
    lk.lock();
    if (rc == AES_OK) mark_issued(s, sl);
  }
}

constexpr uint64_t kInlineIssue = 256;  // batches up to this many requests skip the hand-off
// With no batch on the GPU, batches ramp up: at most kRampBatch requests while no slot is busy,
// four times that with one busy, and so on up to max_batch.  A burst arriving at an idle server
// then reaches the GPU after a small batch's host work instead of a full batch's (descriptor
// building is linear in the batch), and later batches are prepared while earlier ones run.
constexpr uint64_t kRampBatch = 512;

// The worker admits queued requests into batches and retires finished batches.  While a
// batch is in flight it does not sleep: it polls the batches' done events between admissions
// (yielding the core between rounds), so a batch is retired as soon as the GPU has finished
// it; with nothing in flight it keeps polling for cfg.linger_us after its last admission or
// batch (a request that comes within that window finds it awake), then sleeps on cv_work.
void worker_main(aes_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  const double linger = 1e-6 * s->cfg.linger_us;
  double last_active = 0.0;  // last admission or batch on the GPU
  auto idle = [&](bool in_flight) {
    if (in_flight || any_awaiting(s) || (linger > 0.0 && now_s() - last_active < linger)) {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      s->cv_work.wait(lk);
    }
  };
  for (;;) {
    lk.unlock();
    const bool in_flight = poll_completions(s);
    if (in_flight && linger > 0.0) last_active = now_s();
    lk.lock();
    bool any_busy = false;
    int free_slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i) {
      if (s->slots[i].busy) any_busy = true;
      else if (free_slot < 0) free_slot = int(i);
    }
    if (s->stop) {
      // fail whatever is still queued, then wait for the GPU to finish what it has
      for (; s->admit < s->filled; ++s->admit) {
        s->at(s->admit).state.store(AES_REQ_FAILED, std::memory_order_release);
        ++s->failed;
      }
      s->cv_done.notify_all();
      if (!any_busy) break;
      idle(in_flight);
      continue;
    }
    if (free_slot < 0 || s->admit == s->filled) {
      idle(in_flight);
      continue;
    }
    // 2. admit from the head of the queue into one batch: the ticket range [admit, t)
    uint64_t limit = kRampBatch;
    for (const StreamSlot& o : s->slots)
      if (o.busy && limit < s->cfg.max_batch) limit *= 4;
    if (limit > s->cfg.max_batch) limit = s->cfg.max_batch;
    const uint64_t first = s->admit;
    uint64_t t = first;
    while (t < s->filled && t - first < limit && s->inflight < s->cfg.max_inflight) {
      Req& q = s->at(t);
      if (needs_staging(s, q.r)) {
        size_t off = 0;
        if (!s->arena.alloc(q.r.length, &off)) break;  // wait for staging to free up
        q.staged = true;
        q.stage_off = off;
        q.stage_bytes = q.r.length;
      }
      ++s->inflight;
      ++t;
    }
    if (t == first) {
      if (in_flight || any_awaiting(s)) idle(true);
      else if (!any_busy) s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
      else s->cv_work.wait(lk);
      continue;
    }
    s->admit = t;
    if (linger > 0.0) last_active = now_s();
    StreamSlot& sl = s->slots[free_slot];
    sl.busy = true;
    sl.first = first;
    sl.last = t;
    if (s->launches == 0 || s->t_first_launch == 0) s->t_first_launch = now_s();
    ++s->launches;
    s->launched_reqs += t - first;
    sl.inject_fail = s->cfg.fail_every && s->launches % s->cfg.fail_every == 0;  // launches n, 2n, 3n, ...
    if (t - first <= kInlineIssue) {
      // a small batch is issued right here: a hand-off to the issuer thread would cost a
      // thread wake-up, more than the batch's own host work
      lk.unlock();
      const aes_status rc = issue(s, free_slot);
      if (rc != AES_OK) {
        cudaStreamSynchronize(sl.stream);
        retire(s, sl, now_s(), AES_REQ_FAILED);
      }
      lk.lock();
      if (rc == AES_OK) sl.awaiting.store(true, std::memory_order_release);
    } else {
      sl.pending = true;
      s->cv_issue.notify_all();
    }
  }
}

aes_status validate(const aes_server* s, const aes_request* r) {
  if (!r) return set_error(AES_EINVAL, "null request");
  if (r->dir != AES_ENCRYPT && r->dir != AES_DECRYPT) return set_error(AES_EINVAL, "bad dir %u", r->dir);
  if (r->length == 0 || (r->length & 15u)) return set_error(AES_EINVAL, "length must be a positive multiple of 16");
  if (!r->src || !r->dst) return set_error(AES_EINVAL, "null buffer");
  if ((r->src_on_device && (reinterpret_cast<uintptr_t>(r->src) & 15u)) ||
      (r->dst_on_device && (reinterpret_cast<uintptr_t>(r->dst) & 15u)))
    return set_error(AES_EINVAL, "device buffers must be 16-byte aligned");
  if (size_t(r->key_idx) >= s->pool->capacity || s->pool->nr[r->key_idx] == 0)
    return set_error(AES_EINVAL, "key slot %u is not loaded", r->key_idx);
  if (needs_staging(s, *r) && ((r->length + 255) & ~uint64_t(255)) > s->cfg.hbm_budget)
    return set_error(AES_ENOMEM, "request of %llu bytes exceeds the staging budget of %llu bytes",
                     (unsigned long long)r->length, (unsigned long long)s->cfg.hbm_budget);
  return AES_OK;
}

// The checks of validate() without branches on the common path, for bulk submissions:
// validate() runs only when this fails, to name the reason.
inline bool quick_ok(const aes_server* s, const aes_request& r) {
  const uintptr_t mis = ((r.src_on_device ? reinterpret_cast<uintptr_t>(r.src) : 0u) |
                         (r.dst_on_device ? reinterpret_cast<uintptr_t>(r.dst) : 0u)) & 15u;
  const bool key_ok = size_t(r.key_idx) < s->pool->capacity && s->pool->nr[r.key_idx] != 0;
  const bool stage_ok = !needs_staging(s, r) || ((r.length + 255) & ~uint64_t(255)) <= s->cfg.hbm_budget;
  return (r.dir <= 1u) & (r.length != 0) & ((r.length & 15u) == 0) & (r.src != nullptr) & (r.dst != nullptr) &
         (mis == 0) & key_ok & stage_ok;
}

// Writes requests reqs[0..n) as the reserved tickets t0 .. t0+n-1.  The reservation makes the
// slots this thread's alone, so no lock is held; publish() then makes them admissible.
void fill(aes_server* s, uint64_t t0, const aes_request* reqs, size_t n, uint64_t* tickets, double t) {
  for (size_t i = 0; i < n; ++i) {
    const uint64_t tk = t0 + i;
    Req& q = s->at(tk);
    q.r = reqs[i];
    q.t_submit = t;
    q.staged = false;
    q.state.store(AES_REQ_PENDING, std::memory_order_relaxed);
    q.ticket.store(tk, std::memory_order_release);
    tickets[i] = tk;
  }
}

// Moves the fill mark over every ticket now in the ring (a later reservation may have been
// written first).  Holds mu.
void publish(aes_server* s, uint64_t t0, size_t n) {
  if (s->filled == t0) s->filled = t0 + n;
  while (s->filled < s->next_ticket && s->at(s->filled).ticket.load(std::memory_order_acquire) == s->filled) ++s->filled;
}

// Reserves n tickets (room already checked).  Holds mu.
uint64_t reserve(aes_server* s, size_t n, double t) {
  if (s->submitted == 0 || s->t_first == 0) s->t_first = t;
  const uint64_t t0 = s->next_ticket;
  s->next_ticket += n;
  s->submitted += n;
  return t0;
}

// Room for n more tickets: the queue limit, and the ring slots they land on must be free, i.e.
// every older ticket sharing one of those slots has been released (all tickets below `oldest`
// have).  Holds mu.
aes_status room_for(const aes_server* s, size_t n) {
  if (s->next_ticket - s->admit + n > s->cfg.queue_capacity)
    return set_error(AES_EAGAIN, "submission queue full (%u)", s->cfg.queue_capacity);
  if (s->next_ticket + n - 1 >= s->oldest + s->ring_size)
    return set_error(AES_EAGAIN, "no free request slot: poll finished tickets to release them");
  return AES_OK;
}

}  // namespace

using namespace aesgb;

extern "C" {

aes_status aes_server_destroy(aes_server* s) {
  clear_error();
  if (!s) return AES_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();  // returns once no batch is admitted or in flight
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_issuers = true;
  }
  s->cv_issue.notify_all();
  for (std::thread& th : s->issuers)
    if (th.joinable()) th.join();
  for (StreamSlot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.batch) aes_batch_destroy(sl.batch);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
  return AES_OK;
}

aes_status aes_server_create(const aes_server_cfg* cfg, aes_keypool* pool, aes_server** out) {
  clear_error();
  if (!out) return set_error(AES_EINVAL, "null output pointer");
  *out = nullptr;
  if (!cfg || !pool || !pool->entries) return set_error(AES_EINVAL, "null config or key pool");
  if (cfg->hbm_budget < (1u << 20) || cfg->max_inflight == 0 || cfg->nstreams == 0 || cfg->nstreams > 16 ||
      cfg->max_batch == 0 || cfg->max_batch > 65536 || cfg->queue_capacity == 0)
    return set_error(AES_EINVAL, "bad server configuration (budget >= 1 MiB, 1..16 streams, 1..65536 per batch)");
  aes_server* s = new (std::nothrow) aes_server();
  if (!s) return set_error(AES_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->pool = pool;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) { delete s; return cuda_error(e, "cudaGetDevice"); }
  if (s->device != pool->device) { delete s; return set_error(AES_EINVAL, "pool is on another device"); }
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) { delete s; return cuda_error(e, "cudaMemGetInfo"); }
  if (cfg->hbm_budget > free_b) {
    delete s;
    return set_error(AES_ENOMEM, "staging budget %llu exceeds free device memory %zu", (unsigned long long)cfg->hbm_budget, free_b);
  }
  if ((e = cudaMalloc(&s->arena_base, cfg->hbm_budget)) != cudaSuccess) {
    delete s;
    return set_error(AES_ENOMEM, "staging arena cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  s->arena.reset(cfg->hbm_budget);
  {
    const DeviceInfo* di = current_device_info();
    if (!di) {
      aes_server_destroy(s);
      return AES_ECUDA;
    }
    s->host_direct = di->host_direct;
  }
  size_t ring = 1;
  while (ring < cfg->queue_capacity) ring <<= 1;
  try {
    s->ring.reset(new Req[ring]);
    s->lat_us.reserve(std::min<size_t>(ring, kLatencyWindow));
  } catch (...) {
    aes_server_destroy(s);
    return set_error(AES_ENOMEM, "request ring of %zu entries could not be allocated", ring);
  }
  s->mask = ring - 1;
  s->ring_size = ring;
  try {
    for (uint32_t i = 0; i < cfg->nstreams; ++i) s->slots.emplace_back();
    for (StreamSlot& sl : s->slots) {
      sl.lat.reserve(cfg->max_batch);
      sl.frees.reserve(cfg->max_batch);
    }
  } catch (...) {
    aes_server_destroy(s);
    return set_error(AES_ENOMEM, "host allocation failed");
  }
  for (uint32_t i = 0; i < cfg->nstreams; ++i) {
    if ((e = cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking)) != cudaSuccess) {
      aes_server_destroy(s);
      return cuda_error(e, "cudaStreamCreate");
    }
    if ((e = cudaEventCreateWithFlags(&s->slots[i].done_ev, cudaEventDisableTiming)) != cudaSuccess) {
      aes_server_destroy(s);
      return cuda_error(e, "cudaEventCreate");
    }
    aes_status st = aes_batch_create(pool, cfg->max_batch, &s->slots[i].batch);
    if (st != AES_OK) {
      aes_server_destroy(s);
      return st;
    }
  }
  try {
    for (uint32_t i = 0; i < cfg->nstreams; ++i) s->issuers.emplace_back(issuer_main, s, int(i));
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    aes_server_destroy(s);
    return set_error(AES_ENOMEM, "server threads could not be started");
  }
  *out = s;
  return AES_OK;
}

aes_status aes_server_submit(aes_server* s, const aes_request* req, uint64_t* ticket) {
  clear_error();
  if (!s || !ticket) return set_error(AES_EINVAL, "null server or ticket pointer");
  aes_status st = validate(s, req);
  if (st != AES_OK) return st;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(AES_EINVAL, "server is shutting down");
    if ((st = room_for(s, 1)) != AES_OK) return st;
    const double t = now_s();
    const uint64_t t0 = reserve(s, 1, t);
    fill(s, t0, req, 1, ticket, t);
    publish(s, t0, 1);
  }
  s->cv_work.notify_one();
  return AES_OK;
}

aes_status aes_server_submit_many(aes_server* s, const aes_request* reqs, size_t n, uint64_t* tickets) {
  clear_error();
  const double t = now_s();  // the submission starts now, validation included
  if (!s || (n && (!reqs || !tickets))) return set_error(AES_EINVAL, "null server, request or ticket array");
  bool ok = true;
  for (size_t i = 0; i < n; ++i) ok &= quick_ok(s, reqs[i]);
  for (size_t i = 0; !ok && i < n; ++i) {
    aes_status st = validate(s, reqs + i);
    if (st != AES_OK) {
      char why[256];
      std::snprintf(why, sizeof(why), "%s", aes_last_error());
      return set_error(st, "request %zu: %s", i, why);
    }
  }
  if (n == 0) return AES_OK;
  // All n tickets are reserved at once (all or nothing), then written in chunks without the
  // lock; each chunk is published as soon as it is written, so admission and launches start
  // while the rest of the submission is still being written.
  constexpr size_t kChunk = 4096;
  uint64_t t0 = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(AES_EINVAL, "server is shutting down");
    aes_status st = room_for(s, n);
    if (st != AES_OK) return st;
    t0 = reserve(s, n, t);
  }
  for (size_t c = 0; c < n; c += kChunk) {
    const size_t m = std::min(kChunk, n - c);
    fill(s, t0 + c, reqs + c, m, tickets + c, t);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      publish(s, t0 + c, m);
    }
    s->cv_work.notify_one();
  }
  return AES_OK;
}

aes_status aes_server_poll(aes_server* s, uint64_t ticket, int64_t timeout_us, int* state) {
  clear_error();
  if (!s || !state) return set_error(AES_EINVAL, "null server or state pointer");
  std::unique_lock<std::mutex> lk(s->mu);
  auto known = [&] { return ticket != 0 && ticket < s->filled && s->at(ticket).ticket.load(std::memory_order_acquire) == ticket; };
  if (!known()) return set_error(AES_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  auto ready = [&] { return !known() || s->at(ticket).state.load(std::memory_order_acquire) != AES_REQ_PENDING; };
  if (!ready() && timeout_us != 0) {
    if (timeout_us < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  }
  if (!known()) return set_error(AES_ENOTFOUND, "ticket %llu was released by another poll", (unsigned long long)ticket);
  Req& q = s->at(ticket);
  *state = q.state.load(std::memory_order_acquire);
  if (*state == AES_REQ_PENDING) return set_error(AES_ETIMEDOUT, "ticket %llu still pending", (unsigned long long)ticket);
  q.ticket.store(0, std::memory_order_release);  // released: the slot can take a new request
  while (s->oldest < s->filled && s->at(s->oldest).ticket.load(std::memory_order_acquire) != s->oldest) ++s->oldest;
  return AES_OK;
}

aes_status aes_server_stats(aes_server* s, aes_stats* out) {
  clear_error();
  if (!s || !out) return set_error(AES_EINVAL, "null server or output");
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = s->next_ticket - s->admit;
    out->inflight = s->inflight;
    out->launches = s->launches;
    out->bytes_completed = s->bytes_done;
    out->mean_batch = s->launches ? double(s->launched_reqs) / double(s->launches) : 0.0;
    out->gbps = (s->t_last > s->t_first && s->t_first > 0) ? s->bytes_done / (s->t_last - s->t_first) / 1e9 : 0.0;
    out->gbps_from_first_launch = (s->t_last > s->t_first_launch && s->t_first_launch > 0)
                                      ? s->bytes_done / (s->t_last - s->t_first_launch) / 1e9 : 0.0;
    lat = s->lat_us;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      const size_t k = size_t(std::min<double>(lat.size() - 1, std::max(0.0, std::ceil(p * lat.size()) - 1)));
      return lat[k];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = lat.back();
    double sum = 0;
    for (double v : lat) sum += v;
    out->mean_us = sum / lat.size();
  }
  return AES_OK;
}

aes_status aes_server_stats_get(aes_server* s, aes_stats* out) { return aes_server_stats(s, out); }

aes_status aes_server_stats_reset(aes_server* s) {
  clear_error();
  if (!s) return set_error(AES_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_us.clear();
  s->lat_n = 0;
  s->submitted = s->completed = s->failed = s->launches = s->launched_reqs = s->bytes_done = 0;
  s->t_first = s->t_last = s->t_first_launch = 0;
  return AES_OK;
}

}  // extern "C"

extern "C" int aes_testing_arena(size_t size, const int64_t* ops, size_t nops, int64_t* results) {
  if (!ops || !results) return -1;
  Arena a(size);
  std::vector<std::pair<size_t, size_t>> made(nops, {0, 0});  // (offset, bytes) of allocation i
  std::vector<bool> live(nops, false), freed(nops, false);
  for (size_t i = 0; i < nops; ++i) {
    if (ops[i] > 0) {
      size_t off = 0;
      if (a.alloc(size_t(ops[i]), &off)) {
        made[i] = {off, size_t(ops[i])};
        live[i] = true;
        results[i] = int64_t(off);
      } else {
        results[i] = -1;
      }
    } else if (ops[i] < 0) {
      const uint64_t j = uint64_t(-(ops[i] + 1));
      if (j >= i || ops[j] <= 0 || freed[j]) return -1;  // not an earlier allocation, or freed twice
      freed[j] = true;
      if (live[j]) a.release(made[j].first, made[j].second);  // a failed allocation frees nothing
      live[j] = false;
      results[i] = 0;
    } else {
      return -1;
    }
  }
  return 0;
}
