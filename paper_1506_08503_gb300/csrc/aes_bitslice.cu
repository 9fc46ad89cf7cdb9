// aes_bitslice.cu -- the constant-time, gate-level (bitsliced) AES kernel and its launcher;
// the rounds themselves are in aes_bitslice.cuh.
//
// Layout change: a warp loads 1024 consecutive blocks with 128-bit coalesced loads (lane l
// takes blocks l, l+32, ...), and each thread turns its 32 blocks x 128 bits into 128 planes
// with four in-register 32x32 bit transposes (byte permutes for the 16- and 8-bit stages,
// shift+select for the rest); the same transpose turns the planes back before the store.
#include "aes_bitslice.cuh"
#include "aes_internal.cuh"

namespace aesgb {
namespace bs {

__device__ __forceinline__ uint4 ld_block(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_block(uint4* p, uint4 v) {
  asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

constexpr int kThreads = 128;
constexpr int kTile = 1024;  // blocks per warp tile (32 per lane)

// Two CTAs (8 warps) per SM: the 128 planes and the S-box temporaries take up to 255 registers.
// (Three CTAs, 168 registers, spill and measured slower.)  TAIL = false runs whole tiles only
// (nblocks a multiple of kTile), with no bounds checks: their predicates cost registers the
// rounds need (encryption then fits in about 200 registers instead of spilling).  TAIL = true
// is the one ragged last tile (nblocks < kTile), launched apart as a single CTA: absent blocks
// enter as zeros and are not stored.
template <int NR, int DIR, bool TAIL>
__global__ void __launch_bounds__(kThreads, 2) bs_kernel(const uint4* in, uint4* out, size_t nblocks, const Masks km) {
  // the masks go to shared memory, where the rounds' loop reads each column's 32 words as
  // broadcast 16-byte loads
  __shared__ __align__(16) uint32_t msk[(NR + 1) * 128];
  for (int i = threadIdx.x; i < (NR + 1) * 128; i += kThreads) msk[i] = km.m[i >> 7][i & 127];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const size_t warp = (size_t(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const size_t nwarps = (size_t(gridDim.x) * kThreads) >> 5;
  const size_t ntiles = TAIL ? (warp == 0 ? 1 : 0) : nblocks / kTile;
  for (size_t tile = warp; tile < ntiles; tile += nwarps) {
    const size_t base = tile * kTile + lane;
    uint32_t s[128];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const size_t idx = base + 32u * j;
      const uint4 v = (!TAIL || idx < nblocks) ? ld_block(in + idx) : make_uint4(0u, 0u, 0u, 0u);
      s[j] = v.x;
      s[32 + j] = v.y;
      s[64 + j] = v.z;
      s[96 + j] = v.w;
    }
    crypt_tile<NR, DIR>(s, msk);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const size_t idx = base + 32u * j;
      if (!TAIL || idx < nblocks) st_block(out + idx, make_uint4(s[j], s[32 + j], s[64 + j], s[96 + j]));
    }
  }
}

using BSKernel = void (*)(const uint4*, uint4*, size_t, const Masks);

template <bool TAIL>
BSKernel pick(int dir, int nr) {
  if (dir == AES_ENCRYPT) {
    if (nr == 10) return bs_kernel<10, AES_ENCRYPT, TAIL>;
    if (nr == 12) return bs_kernel<12, AES_ENCRYPT, TAIL>;
    if (nr == 14) return bs_kernel<14, AES_ENCRYPT, TAIL>;
  } else {
    if (nr == 10) return bs_kernel<10, AES_DECRYPT, TAIL>;
    if (nr == 12) return bs_kernel<12, AES_DECRYPT, TAIL>;
    if (nr == 14) return bs_kernel<14, AES_DECRYPT, TAIL>;
  }
  return nullptr;
}

}  // namespace bs

aes_status launch_bitslice(int dir, const aes_key_schedule& ks, const uint8_t* iv, const void* d_in,
                           void* d_out, size_t nblocks, cudaStream_t stream, const BSConfig& cfg) {
  (void)cfg;
  bs::BSKernel k = bs::pick<false>(dir, ks.nr), kt = bs::pick<true>(dir, ks.nr);
  if (!k || !kt) return set_error(AES_EINVAL, "no bitsliced kernel for nr=%d", ks.nr);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  bs::Masks km;
  bs::fill_masks(km, ks, dir, iv);
  cudaError_t e;
  const size_t tiles = nblocks / bs::kTile, full = tiles * bs::kTile;
  if (tiles) {
    int per_sm = 0;
    aes_status ast = kernel_ctas_per_sm(reinterpret_cast<const void*>(k), bs::kThreads, 0, &per_sm);
    if (ast != AES_OK) return ast;
    if (per_sm < 1) per_sm = 1;
    const size_t want = (tiles + (bs::kThreads / 32) - 1) / (bs::kThreads / 32);
    const size_t cap = size_t(di->sms) * size_t(per_sm);
    const unsigned grid = unsigned(want < cap ? want : cap);
    k<<<grid, bs::kThreads, 0, stream>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out), full, km);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "bitsliced kernel launch");
  }
  if (nblocks > full) {  // the ragged last tile
    kt<<<1, bs::kThreads, 0, stream>>>(static_cast<const uint4*>(d_in) + full, static_cast<uint4*>(d_out) + full,
                                      nblocks - full, km);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "bitsliced tail launch");
  }
  return AES_OK;
}

}  // namespace aesgb
