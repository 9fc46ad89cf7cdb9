// aes_noalloc.cu -- the batched cipher for callers that must not allocate device memory.
//
// aes_crypt_batched needs a key pool and a batch context, and both allocate device memory.
// Some callers cannot do that: a plug-in whose host application owns every byte of device
// memory and hands out only input and output buffers, or a latency-critical path where
// cudaMalloc is ruled out because it can synchronise the whole device.  This entry point
// keeps all of its working data (the expanded keys, the message descriptors and the block
// starts) in one fixed array in device global memory that the library declares statically,
// so a call allocates nothing: the caller passes its keys, messages, input and output only.
//
// The static array is shared by every call on a device and keeps the last call's contents.
// Nothing in it has to start at zero: each call rewrites every entry its kernels read (keys
// 0..nkeys-1, its own descriptors, block starts and per-warp slices).  Calls issued on the
// SAME stream are safe: the descriptor upload is ordered behind earlier work on that stream.
// Calls that overlap on the GPU (different streams, no synchronisation between them) race on
// the array and may compute with each other's descriptors.  The descriptors are built in one
// shared host buffer, so a call on a stream that is being captured is refused: a graph would
// replay whatever that buffer held last.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "aes_batched.cuh"

namespace {

using namespace aesgb;

constexpr uint32_t kNoAllocMaxKeys = 256;
constexpr uint32_t kNoAllocMaxMsgs = 4096;
constexpr int kThreads = 512, kBlocksPerLane = 2;
constexpr uint32_t kMaxCtas = 256;                         // per direction (one per SM, at most 256)
constexpr uint32_t kMaxWarps = kMaxCtas * (kThreads / 32);  // 4096

struct NoAllocScratch {
  PoolEntry keys[kNoAllocMaxKeys];         // 128 KiB
  BatchMsg msgs[kNoAllocMaxMsgs];          // 128 KiB: encryptions first, then decryptions
  uint64_t start[2][kNoAllocMaxMsgs + 1];  // 64 KiB: block starts per direction
  uint64_t warp_gb[2][kMaxWarps + 1];      // 64 KiB: each warp's first block, slices of equal rounds x blocks
  uint32_t warp_msg[2][kMaxWarps];         // 32 KiB: the message holding that block
};

// Device-side scratch: 416 KiB on every GPU that loads the library, held until exit.  In host
// code this name is only a stand-in; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Host-side staging of the same layout (pageable, in the library's static data), guarded by
// a mutex: one call at a time builds its descriptors here.
NoAllocScratch g_host_stage;
std::mutex g_mu;

constexpr int kMaxDevices = 64;
NoAllocScratch* g_dev_ptr[kMaxDevices] = {nullptr};

// Set-up, once per device with that device current: the scratch's device address.
aes_status scratch_for_current(NoAllocScratch** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(AES_ECUDA, "device ordinal %d out of range", dev);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
      return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_dev_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_dev_ptr[dev];
  return AES_OK;
}

void fill_entry(const aes_key_schedule& ks, PoolEntry& e) {
  std::memset(&e, 0, sizeof(e));
  const KeyWords enc = enc_key_words(ks, nullptr), dec = dec_key_words(ks, nullptr);
  std::memcpy(e.enc, enc.w, sizeof(e.enc));
  std::memcpy(e.dec, dec.w, sizeof(e.dec));
  e.nr = ks.nr;
}

}  // namespace

using namespace aesgb;

extern "C" aes_status aes_crypt_batched_noalloc(const aes_key_schedule* schedules, uint32_t nkeys, const aes_msg* msgs,
                                                size_t nmsgs, const void* d_in, void* d_out, size_t buf_bytes,
                                                void* cuda_stream) {
  clear_error();
  if (nkeys > kNoAllocMaxKeys) return set_error(AES_EINVAL, "%u keys exceed the static maximum of %u", nkeys, kNoAllocMaxKeys);
  if (nmsgs > kNoAllocMaxMsgs) return set_error(AES_EINVAL, "%zu messages exceed the static maximum of %u", nmsgs, kNoAllocMaxMsgs);
  if ((nkeys && !schedules) || (nmsgs && !msgs)) return set_error(AES_EINVAL, "null key or message array");
  for (uint32_t k = 0; k < nkeys; ++k)
    if (!schedule_ok(schedules + k)) return set_error(AES_EINVAL, "key schedule %u is invalid", k);
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), o = reinterpret_cast<uintptr_t>(d_out);
  if (a != o && a < o + buf_bytes && o < a + buf_bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  size_t nenc = 0, ndec = 0;
  for (size_t i = 0; i < nmsgs; ++i) {
    const aes_msg& m = msgs[i];
    if (m.dir != AES_ENCRYPT && m.dir != AES_DECRYPT) return set_error(AES_EINVAL, "message %zu: bad dir %u", i, m.dir);
    if ((m.offset | m.length) & 15u) return set_error(AES_EINVAL, "message %zu: offset and length must be multiples of 16", i);
    if (m.offset > buf_bytes || m.length > buf_bytes - m.offset)
      return set_error(AES_EINVAL, "message %zu leaves the %zu-byte buffers", i, buf_bytes);
    if (m.length == 0) continue;
    if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
    if (m.key_idx >= nkeys) return set_error(AES_EINVAL, "message %zu: key %u of %u", i, m.key_idx, nkeys);
    (m.dir == AES_ENCRYPT ? nenc : ndec)++;
  }
  if (nenc + ndec == 0) return AES_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(AES_EINVAL, "the stream is being captured: this call stages its descriptors in one shared host "
                                 "buffer, so it cannot be recorded into a graph");

  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocScratch* dev = nullptr;
  aes_status st = scratch_for_current(&dev);
  if (st != AES_OK) return st;
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;

  NoAllocScratch& h = g_host_stage;
  int8_t rounds[kNoAllocMaxKeys];
  for (uint32_t k = 0; k < nkeys; ++k) {
    fill_entry(schedules[k], h.keys[k]);
    rounds[k] = int8_t(schedules[k].nr);
  }
  size_t ie = 0, id = nenc;
  uint64_t te = 0, td = 0;
  for (size_t i = 0; i < nmsgs; ++i) {
    const aes_msg& m = msgs[i];
    if (m.length == 0) continue;
    const BatchMsg d{m.key_idx, 0u, m.offset / 16, m.offset / 16, m.length / 16};
    if (m.dir == AES_ENCRYPT) { h.start[0][ie] = te; te += d.nblocks; h.msgs[ie++] = d; }
    else { h.start[1][id - nenc] = td; td += d.nblocks; h.msgs[id++] = d; }
  }
  h.start[0][nenc] = te;
  h.start[1][ndec] = td;

  // Grid per direction: one CTA per SM (at most kMaxCtas), fewer when there is less than one
  // block per thread; every warp gets a slice of equal work in blocks x rounds, so warps
  // holding 14-round messages do not set the kernel's finish time.
  uint32_t grid[2] = {0, 0};
  for (int dir = 0; dir < 2; ++dir) {
    const uint64_t total = dir == AES_ENCRYPT ? te : td;
    if (!total) continue;
    const uint64_t want = (total + kThreads - 1) / kThreads;
    const uint64_t cap_ctas = std::min<uint64_t>(uint64_t(di->sms), kMaxCtas);
    grid[dir] = uint32_t(want < cap_ctas ? want : cap_ctas);
    const BatchMsg* dm = dir == AES_ENCRYPT ? h.msgs : h.msgs + nenc;
    const size_t n = dir == AES_ENCRYPT ? nenc : ndec;
    weighted_slices(dm, h.start[dir], n, rounds, work_of(dm, n, rounds), uint64_t(grid[dir]) * (kThreads / 32),
                    h.warp_gb[dir], h.warp_msg[dir]);
  }

  // Pageable sources: the copies are ordered behind earlier work on `s`, and the staging
  // above may be reused as soon as each copy call returns.
  if ((e = cudaMemcpyAsync(dev->keys, h.keys, nkeys * sizeof(PoolEntry), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dev->msgs, h.msgs, (nenc + ndec) * sizeof(BatchMsg), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dev->start[0], h.start[0], (nenc + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dev->start[1], h.start[1], (ndec + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_error(e, "descriptor upload");
  for (int dir = 0; dir < 2; ++dir) {
    if (!grid[dir]) continue;
    const size_t nw = size_t(grid[dir]) * (kThreads / 32);
    if ((e = cudaMemcpyAsync(dev->warp_gb[dir], h.warp_gb[dir], (nw + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dev->warp_msg[dir], h.warp_msg[dir], nw * sizeof(uint32_t), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
      return cuda_error(e, "slice upload");
  }

  const uint64_t in_base = reinterpret_cast<uint64_t>(d_in), out_base = reinterpret_cast<uint64_t>(d_out);
  for (int dir = 0; dir < 2; ++dir) {
    const uint64_t total = dir == AES_ENCRYPT ? te : td;
    if (!total) continue;
    const BatchDir bd{dir == AES_ENCRYPT ? dev->msgs : dev->msgs + nenc, dev->start[dir], dev->warp_msg[dir], total,
                      uint32_t(dir == AES_ENCRYPT ? nenc : ndec), 0u, dev->warp_gb[dir]};
    const size_t smem = ttable_smem_bytes(dir);
    auto k = dir == AES_ENCRYPT ? tt::tt_batched_kernel<AES_ENCRYPT, kThreads, kBlocksPerLane>
                                : tt::tt_batched_kernel<AES_DECRYPT, kThreads, kBlocksPerLane>;
    {
      aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(k), smem);
      if (ast != AES_OK) return ast;
    }
    k<<<grid[dir], kThreads, smem, s>>>(in_base, out_base, bd, dev->keys);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "batched kernel launch");
  }
  return AES_OK;
}
