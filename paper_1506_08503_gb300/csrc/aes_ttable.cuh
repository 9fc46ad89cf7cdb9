// aes_ttable.cuh -- table-driven AES round kernels (encryption and the equivalent inverse
// cipher) for many independent 16-byte blocks.
//
// One round of the paper's algorithm (Section II: SubBytes, ShiftRows, MixColumns as a
// GF(2^8) matrix product, AddRoundKey; App. A1) is, per output column, the XOR of four
// table words T_j[state byte] and the round-key word, where T_j is the S-box fused with
// column j of circ(2 3 1 1).  Decryption uses the same structure with InvS and
// circ(14 11 13 9) (App. A4) after moving InvMixColumns onto the round keys.
//
// GB300 mapping:
//  * Lookups go to shared memory.  Each of the four tables is replicated 32 times, one copy
//    per bank: entry x of table j for lane l sits at byte offset
//        (j >> 1) * 64 KiB + x * 256 + (j & 1) * 128 + l * 4,
//    so a warp's 32 lookups always hit 32 distinct banks (no conflicts whatever the data),
//    and the address is ONE byte-permute: byte 1 <- state byte, byte 0 <- lane * 4.
//  * Round keys are kernel parameters (constant bank): AddRoundKey is an operand of the
//    same three-input XOR that merges the table words.
//  * Each thread streams blocks with 128-bit loads/stores; consecutive threads take
//    consecutive blocks, so a warp moves 512 contiguous bytes per instruction.
//  * The kernel is persistent (about one CTA per SM, grid-stride over blocks), so the
//    table set-up is paid once per SM per launch.
#pragma once
#include "aes_internal.cuh"

namespace aesgb {

// Each translation unit that includes this header holds its own copy (4.5 KiB).
static __device__ const FieldTables g_field_tables = make_field_tables();

namespace tt {

constexpr uint32_t kRegion = 65536;  // bytes per pair of replicated tables

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int s) {
  return s ? __funnelshift_l(x, x, s) : x;
}

// Byte address of entry (byte k of w) for the calling lane: byte 1 = w.byte[k],
// byte 0 = lane * 4 (from lanec), bytes 2..3 = 0.
template <int K>
__device__ __forceinline__ uint32_t tt_addr(uint32_t w, uint32_t lanec) {
  return __byte_perm(w, lanec, 0x5504u | (K << 4));
}

// Lookup in table J of the entry addressed by byte K of w.
template <int J, int K>
__device__ __forceinline__ uint32_t tt(const char* sm, uint32_t w, uint32_t lanec) {
  constexpr uint32_t off = (J >> 1) * kRegion + (J & 1) * 128u;
  return *reinterpret_cast<const uint32_t*>(sm + tt_addr<K>(w, lanec) + off);
}

// Byte 0 of a, byte 1 of b, byte 2 of c, byte 3 of d.
__device__ __forceinline__ uint32_t pick_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  const uint32_t ab = __byte_perm(a, b, 0x3250u);
  const uint32_t cd = __byte_perm(c, d, 0x7210u);
  return __byte_perm(ab, cd, 0x7610u);
}

template <int DIR>
__device__ __forceinline__ void fill_tables(uint32_t* sm) {
  // Regions 0 and 1: T0|T1 and T2|T3 (rotations of Te0 or Td0).  Region 2 (decryption
  // only): InvS replicated into all four bytes, for the last round.  The 256-entry base
  // tables are staged once (one global read each), then every 16-byte store writes four
  // lanes' copies of one entry.
  __shared__ uint32_t stage[DIR == AES_ENCRYPT ? 256 : 512];
  for (int x = threadIdx.x; x < 256; x += blockDim.x) {
    stage[x] = (DIR == AES_ENCRYPT) ? g_field_tables.te0[x] : g_field_tables.td0[x];
    if (DIR != AES_ENCRYPT) stage[256 + x] = g_field_tables.is4[x];
  }
  __syncthreads();
  constexpr int kVecs = ((DIR == AES_ENCRYPT) ? 2 : 3) * 16384 / 4;
  uint4* sm4 = reinterpret_cast<uint4*>(sm);
  for (int q = threadIdx.x; q < kVecs; q += blockDim.x) {
    const int w = 4 * q;  // first of the four words (lanes 4q..4q+3 of one entry)
    const int region = w >> 14, x = (w >> 6) & 255, half = (w >> 5) & 1;
    const uint32_t v = region < 2 ? rotl32(stage[x], 8 * (2 * region + half)) : (half ? 0u : stage[256 + x]);
    sm4[q] = make_uint4(v, v, v, v);
  }
}

// One middle round on the four column words: encryption takes row i of column c + i through
// T_i (ShiftRows + SubBytes + MixColumns), decryption row i of column c - i through Td_i.
template <int DIR>
__device__ __forceinline__ void tt_round(uint32_t& s0, uint32_t& s1, uint32_t& s2, uint32_t& s3, uint32_t k0,
                                         uint32_t k1, uint32_t k2, uint32_t k3, const char* sm, uint32_t lc) {
  uint32_t t0, t1, t2, t3;
  if constexpr (DIR == AES_ENCRYPT) {
    t0 = tt<0, 0>(sm, s0, lc) ^ tt<1, 1>(sm, s1, lc) ^ tt<2, 2>(sm, s2, lc) ^ tt<3, 3>(sm, s3, lc) ^ k0;
    t1 = tt<0, 0>(sm, s1, lc) ^ tt<1, 1>(sm, s2, lc) ^ tt<2, 2>(sm, s3, lc) ^ tt<3, 3>(sm, s0, lc) ^ k1;
    t2 = tt<0, 0>(sm, s2, lc) ^ tt<1, 1>(sm, s3, lc) ^ tt<2, 2>(sm, s0, lc) ^ tt<3, 3>(sm, s1, lc) ^ k2;
    t3 = tt<0, 0>(sm, s3, lc) ^ tt<1, 1>(sm, s0, lc) ^ tt<2, 2>(sm, s1, lc) ^ tt<3, 3>(sm, s2, lc) ^ k3;
  } else {
    t0 = tt<0, 0>(sm, s0, lc) ^ tt<1, 1>(sm, s3, lc) ^ tt<2, 2>(sm, s2, lc) ^ tt<3, 3>(sm, s1, lc) ^ k0;
    t1 = tt<0, 0>(sm, s1, lc) ^ tt<1, 1>(sm, s0, lc) ^ tt<2, 2>(sm, s3, lc) ^ tt<3, 3>(sm, s2, lc) ^ k1;
    t2 = tt<0, 0>(sm, s2, lc) ^ tt<1, 1>(sm, s1, lc) ^ tt<2, 2>(sm, s0, lc) ^ tt<3, 3>(sm, s3, lc) ^ k2;
    t3 = tt<0, 0>(sm, s3, lc) ^ tt<1, 1>(sm, s2, lc) ^ tt<2, 2>(sm, s1, lc) ^ tt<3, 3>(sm, s0, lc) ^ k3;
  }
  s0 = t0; s1 = t1; s2 = t2; s3 = t3;
}

// Last round (no MixColumns).  Encryption: S(x) is byte 0 of T2 and T3, byte 1 of T3 and T0,
// byte 2 of T0 and T1, byte 3 of T1 and T2.  Decryption: region 2 holds InvS(x) in every byte.
template <int DIR>
__device__ __forceinline__ uint4 tt_final(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3, uint32_t k0,
                                          uint32_t k1, uint32_t k2, uint32_t k3, const char* sm, uint32_t lc) {
  uint4 o;
  if constexpr (DIR == AES_ENCRYPT) {
    o.x = pick_bytes(tt<2, 0>(sm, s0, lc), tt<3, 1>(sm, s1, lc), tt<0, 2>(sm, s2, lc), tt<1, 3>(sm, s3, lc)) ^ k0;
    o.y = pick_bytes(tt<2, 0>(sm, s1, lc), tt<3, 1>(sm, s2, lc), tt<0, 2>(sm, s3, lc), tt<1, 3>(sm, s0, lc)) ^ k1;
    o.z = pick_bytes(tt<2, 0>(sm, s2, lc), tt<3, 1>(sm, s3, lc), tt<0, 2>(sm, s0, lc), tt<1, 3>(sm, s1, lc)) ^ k2;
    o.w = pick_bytes(tt<2, 0>(sm, s3, lc), tt<3, 1>(sm, s0, lc), tt<0, 2>(sm, s1, lc), tt<1, 3>(sm, s2, lc)) ^ k3;
  } else {
    o.x = pick_bytes(tt<4, 0>(sm, s0, lc), tt<4, 1>(sm, s3, lc), tt<4, 2>(sm, s2, lc), tt<4, 3>(sm, s1, lc)) ^ k0;
    o.y = pick_bytes(tt<4, 0>(sm, s1, lc), tt<4, 1>(sm, s0, lc), tt<4, 2>(sm, s3, lc), tt<4, 3>(sm, s2, lc)) ^ k1;
    o.z = pick_bytes(tt<4, 0>(sm, s2, lc), tt<4, 1>(sm, s1, lc), tt<4, 2>(sm, s0, lc), tt<4, 3>(sm, s3, lc)) ^ k2;
    o.w = pick_bytes(tt<4, 0>(sm, s3, lc), tt<4, 1>(sm, s2, lc), tt<4, 2>(sm, s1, lc), tt<4, 3>(sm, s0, lc)) ^ k3;
  }
  return o;
}

// A whole block with NR rounds and the round keys in the constant bank (kernel parameter).
template <int NR, int DIR>
__device__ __forceinline__ uint4 crypt_block(uint4 v, const KeyWords& kw, const char* sm, uint32_t lc) {
  uint32_t s0 = v.x ^ kw.w[0][0], s1 = v.y ^ kw.w[0][1], s2 = v.z ^ kw.w[0][2], s3 = v.w ^ kw.w[0][3];
#pragma unroll
  for (int r = 1; r < NR; ++r) tt_round<DIR>(s0, s1, s2, s3, kw.w[r][0], kw.w[r][1], kw.w[r][2], kw.w[r][3], sm, lc);
  return tt_final<DIR>(s0, s1, s2, s3, kw.w[NR][0], kw.w[NR][1], kw.w[NR][2], kw.w[NR][3], sm, lc);
}

__device__ __forceinline__ uint4 ld_block(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

// Asks L2 to fetch the line holding p (no register result, no fault on any address).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}

__device__ __forceinline__ void st_block(uint4* p, uint4 v) {
  asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// ---- four lanes per block (CBC encryption chains, where latency is the bound) ----------------
// Lane q of an aligned group of four holds column q of the state.  Byte i of column q feeds
// output column q - i through T_i, so each lane looks up its own four bytes at once and the
// three words bound for other columns move to their lanes by shuffles inside the group:
// per round one byte permute + lookup, one shuffle and two XORs on the dependent path.
__device__ __forceinline__ uint32_t group_shfl(uint32_t v, uint32_t lane, uint32_t d) {
  return __shfl_sync(0xFu << (lane & ~3u), v, (lane & ~3u) | ((lane + d) & 3u));
}

// One middle encryption round of column lane & 3 with its round-key word k.
__device__ __forceinline__ uint32_t col_round(uint32_t s, uint32_t k, const char* sm, uint32_t lane, uint32_t lc) {
  const uint32_t a1 = tt<1, 1>(sm, s, lc), a2 = tt<2, 2>(sm, s, lc), a3 = tt<3, 3>(sm, s, lc);
  const uint32_t a0 = tt<0, 0>(sm, s, lc);
  return a0 ^ group_shfl(a1, lane, 1) ^ group_shfl(a2, lane, 2) ^ group_shfl(a3, lane, 3) ^ k;
}

// The last encryption round before its AddRoundKey (S-box bytes picked out of the table
// words, as in tt_final); the caller adds the last round key.
__device__ __forceinline__ uint32_t col_last(uint32_t s, const char* sm, uint32_t lane, uint32_t lc) {
  const uint32_t b1 = tt<3, 1>(sm, s, lc), b2 = tt<0, 2>(sm, s, lc), b3 = tt<1, 3>(sm, s, lc);
  const uint32_t b0 = tt<2, 0>(sm, s, lc);
  return pick_bytes(b0, group_shfl(b1, lane, 1), group_shfl(b2, lane, 2), group_shfl(b3, lane, 3));
}

template <int NR, int DIR, int THREADS, int U>
__global__ void __launch_bounds__(THREADS, 1)
tt_kernel(const uint4* in, uint4* out, size_t nblocks, const KeyWords kw) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<DIR>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lc = (threadIdx.x & 31u) * 4u;
  const size_t stride = size_t(gridDim.x) * THREADS;
  size_t i = size_t(blockIdx.x) * THREADS + threadIdx.x;
  for (; i + (U - 1) * stride < nblocks; i += U * stride) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_block(in + i + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u)  // the next iteration's blocks, while this one computes
      if (i + (U + u) * stride < nblocks) prefetch_l2(in + i + (U + u) * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = crypt_block<NR, DIR>(v[u], kw, sm, lc);
#pragma unroll
    for (int u = 0; u < U; ++u) st_block(out + i + u * stride, v[u]);
  }
  for (; i < nblocks; i += stride) st_block(out + i, crypt_block<NR, DIR>(ld_block(in + i), kw, sm, lc));
}

// The configurations (CTA size, blocks in flight per thread) the autotuner may pick from.
// 1024-thread CTAs are limited to 64 registers, so they take at most two blocks in flight.
template <int NR, int DIR>
TTKernelFn select_config(int threads, int unroll) {
  if (threads == 256 && unroll == 4) return tt_kernel<NR, DIR, 256, 4>;
  if (threads == 512 && unroll == 1) return tt_kernel<NR, DIR, 512, 1>;
  if (threads == 512 && unroll == 2) return tt_kernel<NR, DIR, 512, 2>;
  if (threads == 512 && unroll == 4) return tt_kernel<NR, DIR, 512, 4>;
  if (threads == 768 && unroll == 2) return tt_kernel<NR, DIR, 768, 2>;
  if (threads == 1024 && unroll == 1) return tt_kernel<NR, DIR, 1024, 1>;
  if (threads == 1024 && unroll == 2) return tt_kernel<NR, DIR, 1024, 2>;
  return nullptr;
}

}  // namespace tt
}  // namespace aesgb
