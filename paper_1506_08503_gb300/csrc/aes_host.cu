// aes_host.cu -- encryption/decryption of HOST buffers.
//
// Where kernels may load and store host memory themselves (pageable access through the host
// page tables, as Grace-Blackwell offers over NVLink-C2C) and both buffers are 16-byte
// aligned, the cipher kernel runs on the host buffers directly: every byte crosses the link
// once in each direction, as with copies, but without staging or copy engines (measured on a
// GB300: 170 GB/s each way against 144-157 GB/s for the copy pipeline).  Otherwise the library
// stages the data through device memory in chunks, overlapping host->device copies, the
// cipher kernel and device->host copies on three streams.
#include <cstring>
#include <mutex>

#include "aes_internal.cuh"

namespace aesgb {
namespace {

constexpr int kSlots = 3;
constexpr size_t kChunkBytes = size_t(64) << 20;  // 64 MiB per slot

struct Staging {
  int device = -1;
  void* buf[kSlots] = {nullptr, nullptr, nullptr};
  cudaStream_t stream[kSlots] = {nullptr, nullptr, nullptr};
  cudaEvent_t done[kSlots] = {nullptr, nullptr, nullptr};
  cudaEvent_t start = nullptr;
  std::mutex mu;  // one host-buffer call at a time per device
};

constexpr int kMaxDevices = 64;
Staging g_stage[kMaxDevices];
std::mutex g_stage_mu;

aes_status staging_for_current(Staging** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(AES_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_stage_mu);
  Staging& s = g_stage[dev];
  if (s.device != dev) {
    for (int i = 0; i < kSlots; ++i) {
      if ((e = cudaMalloc(&s.buf[i], kChunkBytes)) != cudaSuccess) return set_error(AES_ENOMEM, "staging cudaMalloc failed: %s", cudaGetErrorString(e));
      if ((e = cudaStreamCreateWithFlags(&s.stream[i], cudaStreamNonBlocking)) != cudaSuccess) return cuda_error(e, "cudaStreamCreate");
      if ((e = cudaEventCreateWithFlags(&s.done[i], cudaEventDisableTiming)) != cudaSuccess) return cuda_error(e, "cudaEventCreate");
    }
    if ((e = cudaEventCreateWithFlags(&s.start, cudaEventDisableTiming)) != cudaSuccess) return cuda_error(e, "cudaEventCreate");
    s.device = dev;
  }
  *out = &s;
  return AES_OK;
}

}  // namespace
}  // namespace aesgb

using namespace aesgb;

extern "C" aes_status aes_crypt_host(const aes_key_schedule* ks, const uint8_t* iv, const void* h_in,
                                     void* h_out, size_t nblocks, int dir, int impl, void* cuda_stream) {
  clear_error();
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (impl != AES_IMPL_AUTO && impl != AES_IMPL_TTABLE && impl != AES_IMPL_BITSLICE)
    return set_error(AES_EINVAL, "unknown impl %d", impl);
  if (nblocks == 0) return AES_OK;
  if (!h_in || !h_out) return set_error(AES_EINVAL, "null buffer");
  if (nblocks > (SIZE_MAX >> 5)) return set_error(AES_EINVAL, "nblocks too large");
  const uintptr_t a = reinterpret_cast<uintptr_t>(h_in), b = reinterpret_cast<uintptr_t>(h_out);
  const uintptr_t bytes = uintptr_t(nblocks) * 16u;
  if (a != b && a < b + bytes && b < a + bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");

  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  if (di->host_direct && ((a | b) & 15u) == 0) {
    aes_status st = aes_crypt_blocks(ks, iv, h_in, h_out, nblocks, dir, impl, cuda_stream);
    if (st != AES_OK) return st;
    const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? AES_OK : cuda_error(e, "host-buffer kernel");
  }
  Staging* s = nullptr;
  aes_status st = staging_for_current(&s);
  if (st != AES_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  const KeyWords kw = dir == AES_ENCRYPT ? enc_key_words(*ks, iv) : dec_key_words(*ks, iv);
  cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaEventRecord(s->start, user);  // order after the caller's prior work
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  for (int i = 0; i < kSlots; ++i)
    if ((e = cudaStreamWaitEvent(s->stream[i], s->start, 0)) != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");

  const size_t chunk_blocks = kChunkBytes / 16;
  const char* src = static_cast<const char*>(h_in);
  char* dst = static_cast<char*>(h_out);
  size_t done = 0;
  for (size_t c = 0; done < nblocks; ++c) {
    const int slot = int(c % kSlots);
    cudaStream_t str = s->stream[slot];
    const size_t n = (nblocks - done) < chunk_blocks ? (nblocks - done) : chunk_blocks;
    // stream order makes the slot's previous D2H finish before this H2D overwrites it
    if ((e = cudaMemcpyAsync(s->buf[slot], src + done * 16, n * 16, cudaMemcpyHostToDevice, str)) != cudaSuccess)
      return cuda_error(e, "cudaMemcpyAsync H2D");
    if (impl == AES_IMPL_BITSLICE) st = launch_bitslice(dir, *ks, iv, s->buf[slot], s->buf[slot], n, str, BSConfig{});
    else st = launch_ttable(dir, ks->nr, kw, s->buf[slot], s->buf[slot], n, str, TTConfig{});
    if (st != AES_OK) return st;
    if ((e = cudaMemcpyAsync(dst + done * 16, s->buf[slot], n * 16, cudaMemcpyDeviceToHost, str)) != cudaSuccess)
      return cuda_error(e, "cudaMemcpyAsync D2H");
    done += n;
  }
  for (int i = 0; i < kSlots; ++i) {
    if ((e = cudaEventRecord(s->done[i], s->stream[i])) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    if ((e = cudaEventSynchronize(s->done[i])) != cudaSuccess) return cuda_error(e, "host-buffer pipeline");
  }
  return AES_OK;
}
