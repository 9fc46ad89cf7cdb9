// aes_ctr_scan.cu -- two follow-ons of the independent-block kernel.
//
// Counter mode.  The paper names counter-based modes (GCM) as future work (Section V); the
// counter part needs no new field arithmetic: block i is P_i xor E(T + i), where T is the
// initial 128-bit counter block read as a big-endian integer and the addition is mod 2^128 (the
// usual counter increment).  Encryption and decryption are the same operation.  Every block is
// independent, so it runs like the independent-block kernel; the counter is formed in
// registers and the data costs one load and one store per block.
//
// Equality scan over a deterministically encrypted column.  The paper's motivation is queries
// on encrypted database columns (Section I): under one key and IV, equal 16-byte records give
// equal ciphertexts, so an equality query is a scan for the query's ciphertext.  The scan
// reads 16 bytes per record once (bound by HBM, not by the cipher) and appends matching record
// indices through one atomic counter per warp with matches.
#include <cstring>

#include "aes_ttable.cuh"

namespace aesgb {
namespace {

using namespace tt;

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123u); }

// Counter block T + i as the four little-endian state words of its bytes (big-endian integer).
__device__ __forceinline__ uint4 counter_block(uint64_t hi, uint64_t lo, uint64_t i) {
  const uint64_t l = lo + i;
  const uint64_t h = hi + (l < lo ? 1u : 0u);
  return make_uint4(bswap32(uint32_t(h >> 32)), bswap32(uint32_t(h)), bswap32(uint32_t(l >> 32)), bswap32(uint32_t(l)));
}

// 24 warps per SM, as in the tuned independent-block kernel (the 128 KiB of tables allow one
// CTA per SM, so the CTA takes the warps)
constexpr unsigned kCtrThreads = 768;

template <int NR>
__global__ void __launch_bounds__(kCtrThreads, 1)
ctr_kernel(const uint4* in, uint4* out, size_t nblocks, uint64_t ctr_hi, uint64_t ctr_lo, const KeyWords kw) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lc = (threadIdx.x & 31u) * 4u;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  // two blocks in flight per thread, as in the independent-block kernel
  for (; i + stride < nblocks; i += 2 * stride) {
    const uint4 p0 = ld_block(in + i), p1 = ld_block(in + i + stride);
    const uint4 k0 = crypt_block<NR, AES_ENCRYPT>(counter_block(ctr_hi, ctr_lo, i), kw, sm, lc);
    const uint4 k1 = crypt_block<NR, AES_ENCRYPT>(counter_block(ctr_hi, ctr_lo, i + stride), kw, sm, lc);
    st_block(out + i, make_uint4(p0.x ^ k0.x, p0.y ^ k0.y, p0.z ^ k0.z, p0.w ^ k0.w));
    st_block(out + i + stride, make_uint4(p1.x ^ k1.x, p1.y ^ k1.y, p1.z ^ k1.z, p1.w ^ k1.w));
  }
  if (i < nblocks) {
    const uint4 p = ld_block(in + i);
    const uint4 k = crypt_block<NR, AES_ENCRYPT>(counter_block(ctr_hi, ctr_lo, i), kw, sm, lc);
    st_block(out + i, make_uint4(p.x ^ k.x, p.y ^ k.y, p.z ^ k.z, p.w ^ k.w));
  }
}

// HBM-bound: each thread issues kScanU independent 16-byte loads before it compares any, so
// that more bytes are in flight per SM; loads at u * stride keep every warp instruction on 512
// contiguous bytes.  Measured on one GB300, 10^7 records, 20 calls back to back: one load per
// step 30.5-30.7 us per call, two 27.6-28.1, four 28.9-29.0 (eight per warp, contiguous, as two).
constexpr int kScanU = 2;

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__global__ void __launch_bounds__(256)
scan_equal_kernel(const uint4* col, size_t n, uint4 needle, unsigned long long* matches, size_t max_matches,
                  unsigned long long* count) {
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u;
  // every lane of the warp runs the same number of iterations (the bound is tested on the
  // warp's first index), so each ballot is warp-wide
  const size_t n_round = (n + 31) & ~size_t(31);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i - lane < n_round; i += kScanU * stride) {
    uint4 v[kScanU];
#pragma unroll
    for (int u = 0; u < kScanU; ++u) {
      const size_t j = i + u * stride;
      v[u] = j < n ? ld_stream(col + j) : make_uint4(~needle.x, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kScanU; ++u) {
      const size_t j = i + u * stride;
      const bool hit = j < n && v[u].x == needle.x && v[u].y == needle.y && v[u].z == needle.z && v[u].w == needle.w;
      const uint32_t mask = __ballot_sync(0xFFFFFFFFu, hit);
      if (mask) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (hit) {
          const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
          if (slot < max_matches) matches[slot] = j;
        }
      }
    }
  }
}

using CtrKernel = void (*)(const uint4*, uint4*, size_t, uint64_t, uint64_t, const KeyWords);

}  // namespace
}  // namespace aesgb

using namespace aesgb;

extern "C" aes_status aes_ctr_crypt(const aes_key_schedule* ks, const uint8_t* ctr0, const void* d_in, void* d_out,
                                    size_t nblocks, void* cuda_stream) {
  clear_error();
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (!ctr0) return set_error(AES_EINVAL, "null counter block");
  if (nblocks == 0) return AES_OK;
  if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  if (nblocks > (SIZE_MAX >> 5)) return set_error(AES_EINVAL, "nblocks too large");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  const uintptr_t bytes = uintptr_t(nblocks) * 16u;
  if (a != b && a < b + bytes && b < a + bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  uint64_t hi = 0, lo = 0;
  for (int i = 0; i < 8; ++i) {
    hi = (hi << 8) | ctr0[i];
    lo = (lo << 8) | ctr0[8 + i];
  }
  const KeyWords kw = enc_key_words(*ks, nullptr);
  CtrKernel k = ks->nr == 10 ? ctr_kernel<10> : ks->nr == 12 ? ctr_kernel<12> : ctr_kernel<14>;
  const size_t smem = ttable_smem_bytes(AES_ENCRYPT);
  aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(k), smem);
  if (ast != AES_OK) return ast;
  cudaError_t e;
  const size_t want = (nblocks + kCtrThreads - 1) / kCtrThreads;
  const unsigned grid = unsigned(want < size_t(di->sms) ? want : size_t(di->sms));
  k<<<grid, kCtrThreads, smem, static_cast<cudaStream_t>(cuda_stream)>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                                                 nblocks, hi, lo, kw);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CTR kernel launch");
  return AES_OK;
}

extern "C" aes_status aes_scan_equal(const void* d_column, size_t nrecords, const uint8_t* needle, uint64_t* d_matches,
                                     size_t max_matches, uint64_t* d_count, void* cuda_stream) {
  clear_error();
  if (!needle || !d_count) return set_error(AES_EINVAL, "null needle or count");
  if (max_matches && !d_matches) return set_error(AES_EINVAL, "null match array");
  if ((reinterpret_cast<uintptr_t>(d_column) & 15u) || (reinterpret_cast<uintptr_t>(d_count) & 7u) ||
      (reinterpret_cast<uintptr_t>(d_matches) & 7u))
    return set_error(AES_EINVAL, "column must be 16-byte aligned, counters and indices 8-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(count)");
  if (nrecords == 0) return AES_OK;
  if (!d_column) return set_error(AES_EINVAL, "null column");
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  uint4 nd;
  std::memcpy(&nd, needle, 16);
  const size_t want = (nrecords + 255) / 256;
  const size_t cap = size_t(di->sms) * 8;
  const unsigned grid = unsigned(want < cap ? want : cap);
  scan_equal_kernel<<<grid, 256, 0, st>>>(static_cast<const uint4*>(d_column), nrecords, nd,
                                          reinterpret_cast<unsigned long long*>(d_matches), max_matches,
                                          reinterpret_cast<unsigned long long*>(d_count));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "scan kernel launch");
  return AES_OK;
}
