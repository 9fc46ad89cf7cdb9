// aes_bitslice.cu -- constant-time, gate-level (bitsliced) AES kernels.
//
// The paper computes SubBytes as GF(2^8) inversion plus an affine map and MixColumns as a
// GF(2^8) matrix product (Section II, App. A1-A5).  Here both are Boolean circuits evaluated
// on "planes": each thread owns 32 blocks, and its 128 registers s[8b + i] hold bit i of
// state byte b for all 32 blocks (bit j of a plane = block j).  Then
//   * SubBytes is the tower-field S-box circuit (aes_bitslice_sbox.cuh) on 8 planes, 16 times;
//   * ShiftRows is a renaming of registers (no instruction);
//   * MixColumns is an XOR network: out_r = xtime(a_r ^ a_r+1) ^ a_r+1 ^ a_r+2 ^ a_r+3, where
//     xtime on planes moves plane 7 into planes 0, 1, 3, 4;
//   * InvMixColumns = MixColumns o P with P(col)_r = a_r ^ 4 (a_r ^ a_r+2), since
//     circ(14,11,13,9) = circ(2,3,1,1) * circ(5,0,4,0) over GF(2^8);
//   * AddRoundKey XORs each plane with an all-zeros or all-ones mask held in the constant
//     bank (kernel parameter), so the key costs no memory traffic.
// No table, no data-dependent branch or address: time is independent of data and key.
//
// Layout change: a warp loads 1024 consecutive blocks with 128-bit coalesced loads (lane l
// takes blocks l, l+32, ...), and each thread turns its 32 blocks x 128 bits into 128 planes
// with four in-register 32x32 bit transposes (byte permutes for the 16- and 8-bit stages,
// shift+select for the rest); the same transpose turns the planes back before the store.
#include "aes_bitslice_sbox.cuh"
#include "aes_internal.cuh"

namespace aesgb {
namespace bs {

struct Masks {
  uint32_t m[kMaxRounds + 1][128];
};

// 32x32 bit transpose in place: afterwards bit j of a[p] is the old bit p of a[j].
__device__ __forceinline__ void transpose32(uint32_t* a) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t x = a[k], y = a[k + 16];
    a[k] = __byte_perm(x, y, 0x5410u);
    a[k + 16] = __byte_perm(x, y, 0x7632u);
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k & 8) continue;
    const uint32_t x = a[k], y = a[k + 8];
    a[k] = __byte_perm(x, y, 0x6240u);
    a[k + 8] = __byte_perm(x, y, 0x7351u);
  }
#pragma unroll
  for (int j = 4; j >= 1; j >>= 1) {
    const uint32_t m = j == 4 ? 0x0F0F0F0Fu : j == 2 ? 0x33333333u : 0x55555555u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const uint32_t x = a[k], y = a[k + j];
      a[k] = (x & m) | ((y << j) & ~m);
      a[k + j] = (y & ~m) | ((x >> j) & m);
    }
  }
}

// xtime (multiplication by x) of one bitsliced byte
__device__ __forceinline__ void xtime8(const uint32_t* u, uint32_t* v) {
  v[0] = u[7];
  v[1] = u[0] ^ u[7];
  v[2] = u[1];
  v[3] = u[2] ^ u[7];
  v[4] = u[3] ^ u[7];
  v[5] = u[4];
  v[6] = u[5];
  v[7] = u[6];
}

__device__ __forceinline__ void ark(uint32_t* s, const uint32_t* k) {
#pragma unroll
  for (int i = 0; i < 128; ++i) s[i] ^= k[i];
}

__device__ __forceinline__ void sub_bytes(uint32_t* s) {
#pragma unroll
  for (int b = 0; b < 16; ++b) sbox_planes(s[8 * b], s[8 * b + 1], s[8 * b + 2], s[8 * b + 3], s[8 * b + 4], s[8 * b + 5], s[8 * b + 6], s[8 * b + 7]);
}

__device__ __forceinline__ void inv_sub_bytes(uint32_t* s) {
#pragma unroll
  for (int b = 0; b < 16; ++b) inv_sbox_planes(s[8 * b], s[8 * b + 1], s[8 * b + 2], s[8 * b + 3], s[8 * b + 4], s[8 * b + 5], s[8 * b + 6], s[8 * b + 7]);
}

// byte (r, c) of the state is byte r + 4c; ShiftRows reads row r of column c + r
__device__ __forceinline__ constexpr int sr_src(int r, int c) { return r + 4 * ((c + r) & 3); }
__device__ __forceinline__ constexpr int isr_src(int r, int c) { return r + 4 * ((c - r) & 3); }

// ShiftRows then MixColumns (rounds 1..Nr-1) or ShiftRows alone (last round), into n.
template <bool MIX>
__device__ __forceinline__ void shift_mix(const uint32_t* s, uint32_t* n) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!MIX) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = s[8 * sr_src(r, c) + i];
      continue;
    }
    const uint32_t* a[4] = {s + 8 * sr_src(0, c), s + 8 * sr_src(1, c), s + 8 * sr_src(2, c), s + 8 * sr_src(3, c)};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t t[8], x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) t[i] = a[r][i] ^ a[(r + 1) & 3][i];
      xtime8(t, x);
#pragma unroll
      for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = x[i] ^ a[(r + 1) & 3][i] ^ a[(r + 2) & 3][i] ^ a[(r + 3) & 3][i];
    }
  }
}

// InvMixColumns in place on every column (no shift): MixColumns o P.
__device__ __forceinline__ void inv_mix(uint32_t* s) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t* a[4] = {s + 8 * (4 * c), s + 8 * (4 * c + 1), s + 8 * (4 * c + 2), s + 8 * (4 * c + 3)};
    uint32_t b[4][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // P: b_r = a_r ^ 4 (a_r ^ a_r+2); the two pairs share u
      uint32_t u[8], v[8], w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) u[i] = a[h][i] ^ a[h + 2][i];
      xtime8(u, v);
      xtime8(v, w);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        b[h][i] = a[h][i] ^ w[i];
        b[h + 2][i] = a[h + 2][i] ^ w[i];
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      uint32_t t[8], x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) t[i] = b[r][i] ^ b[(r + 1) & 3][i];
      xtime8(t, x);
#pragma unroll
      for (int i = 0; i < 8; ++i) a[r][i] = x[i] ^ b[(r + 1) & 3][i] ^ b[(r + 2) & 3][i] ^ b[(r + 3) & 3][i];
    }
  }
}

__device__ __forceinline__ void inv_shift(const uint32_t* s, uint32_t* n) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = s[8 * isr_src(r, c) + i];
}

template <int NR>
__device__ __forceinline__ void encrypt_planes(uint32_t* s, const Masks& km) {
  ark(s, km.m[0]);
#pragma unroll
  for (int r = 1; r <= NR; ++r) {
    sub_bytes(s);
    uint32_t n[128];
    if (r < NR) shift_mix<true>(s, n);
    else shift_mix<false>(s, n);
#pragma unroll
    for (int i = 0; i < 128; ++i) s[i] = n[i] ^ km.m[r][i];
  }
}

// The paper's inverse cipher order (App. A4): for r = Nr..1 add K_r, InvMixColumns unless
// r = Nr, InvShiftRows, InvSubBytes; then add K_0 (which carries the IV).
template <int NR>
__device__ __forceinline__ void decrypt_planes(uint32_t* s, const Masks& km) {
#pragma unroll
  for (int r = NR; r >= 1; --r) {
    ark(s, km.m[r]);
    if (r < NR) inv_mix(s);
    uint32_t n[128];
    inv_shift(s, n);
#pragma unroll
    for (int i = 0; i < 128; ++i) s[i] = n[i];
    inv_sub_bytes(s);
  }
  ark(s, km.m[0]);
}

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

template <int NR, int DIR>
__global__ void __launch_bounds__(kThreads) bs_kernel(const uint4* in, uint4* out, size_t nblocks, const Masks km) {
  const unsigned lane = threadIdx.x & 31u;
  const size_t warp = (size_t(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const size_t nwarps = (size_t(gridDim.x) * kThreads) >> 5;
  const size_t ntiles = (nblocks + kTile - 1) / kTile;
  for (size_t tile = warp; tile < ntiles; tile += nwarps) {
    const size_t base = tile * kTile + lane;
    uint32_t s[128];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const size_t idx = base + 32u * j;
      const uint4 v = idx < nblocks ? ld_block(in + idx) : make_uint4(0u, 0u, 0u, 0u);
      s[j] = v.x;
      s[32 + j] = v.y;
      s[64 + j] = v.z;
      s[96 + j] = v.w;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) transpose32(s + 32 * q);
    if constexpr (DIR == AES_ENCRYPT) encrypt_planes<NR>(s, km);
    else decrypt_planes<NR>(s, km);
#pragma unroll
    for (int q = 0; q < 4; ++q) transpose32(s + 32 * q);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const size_t idx = base + 32u * j;
      if (idx < nblocks) st_block(out + idx, make_uint4(s[j], s[32 + j], s[64 + j], s[96 + j]));
    }
  }
}

using BSKernel = void (*)(const uint4*, uint4*, size_t, const Masks);

BSKernel pick(int dir, int nr) {
  if (dir == AES_ENCRYPT) {
    if (nr == 10) return bs_kernel<10, AES_ENCRYPT>;
    if (nr == 12) return bs_kernel<12, AES_ENCRYPT>;
    if (nr == 14) return bs_kernel<14, AES_ENCRYPT>;
  } else {
    if (nr == 10) return bs_kernel<10, AES_DECRYPT>;
    if (nr == 12) return bs_kernel<12, AES_DECRYPT>;
    if (nr == 14) return bs_kernel<14, AES_DECRYPT>;
  }
  return nullptr;
}

void fill_masks(Masks& km, const aes_key_schedule& ks, int r, const uint8_t* extra) {
  for (int b = 0; b < 16; ++b) {
    const uint8_t k = uint8_t(ks.rk[r][b] ^ (extra ? extra[b] : 0));
    for (int i = 0; i < 8; ++i) km.m[r][8 * b + i] = ((k >> i) & 1u) ? 0xFFFFFFFFu : 0u;
  }
}

}  // namespace bs

aes_status launch_bitslice(int dir, const aes_key_schedule& ks, const uint8_t* iv, const void* d_in,
                           void* d_out, size_t nblocks, cudaStream_t stream, const BSConfig& cfg) {
  (void)cfg;
  bs::BSKernel k = bs::pick(dir, ks.nr);
  if (!k) return set_error(AES_EINVAL, "no bitsliced kernel for nr=%d", ks.nr);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  bs::Masks km;
  for (int r = 0; r <= ks.nr; ++r) bs::fill_masks(km, ks, r, r == 0 ? iv : nullptr);  // IV rides on K0
  int per_sm = 0;
  aes_status ast = kernel_ctas_per_sm(reinterpret_cast<const void*>(k), bs::kThreads, 0, &per_sm);
  if (ast != AES_OK) return ast;
  cudaError_t e;
  if (per_sm < 1) per_sm = 1;
  const size_t tiles = (nblocks + bs::kTile - 1) / bs::kTile;
  const size_t want = (tiles + (bs::kThreads / 32) - 1) / (bs::kThreads / 32);
  const size_t cap = size_t(di->sms) * size_t(per_sm);
  const unsigned grid = unsigned(want < cap ? want : cap);
  k<<<grid, bs::kThreads, 0, stream>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out), nblocks, km);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "bitsliced kernel launch");
  return AES_OK;
}

}  // namespace aesgb
