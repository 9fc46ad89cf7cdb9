// aes_small.cu -- the T-table rounds for small calls, with the tables read from global memory.
//
// The shared-memory kernel (aes_ttable.cuh) fills 128-192 KiB of replicated tables in every
// CTA before its first lookup: the right trade when each CTA then enciphers thousands of
// blocks, most of a call's time when a call holds a few thousand blocks in all.  Here the four
// round tables (rotations of the fused S-box and MixColumns table, App. A1; for decryption the
// InvS and InvMixColumns table, App. A4) and the last round's S-box word sit in one 10 KiB
// device array built at compile time from the field, read through the read-only cache: no
// fill, one 16-byte block per thread, as many CTAs as the blocks need.  The lookups of a warp
// may meet in one cache bank (the replicated shared-memory layout avoids that), which costs
// throughput the latency-bound small call does not need.
#include "aes_ttable.cuh"

namespace aesgb {
namespace {

struct SmallTables {
  uint32_t te[4][256];  // te[j][x] = Te0[x] rotated left by 8j bits (row j of column j's table)
  uint32_t s4[256];     // S(x) in all four bytes
  uint32_t td[4][256];
  uint32_t is4[256];
};

AES_HD constexpr uint32_t rotl_c(uint32_t x, int s) { return s ? (x << s) | (x >> (32 - s)) : x; }

AES_HD constexpr SmallTables make_small_tables() {
  SmallTables t{};
  const FieldTables f = make_field_tables();
  for (int x = 0; x < 256; ++x) {
    for (int j = 0; j < 4; ++j) {
      t.te[j][x] = rotl_c(f.te0[x], 8 * j);
      t.td[j][x] = rotl_c(f.td0[x], 8 * j);
    }
    t.s4[x] = f.s4[x];
    t.is4[x] = f.is4[x];
  }
  return t;
}

__device__ const SmallTables g_small = make_small_tables();

template <int K>
__device__ __forceinline__ uint32_t byte_of(uint32_t w) { return (w >> (8 * K)) & 0xFFu; }

template <int J, int K>
__device__ __forceinline__ uint32_t gl(const uint32_t (&t)[4][256], uint32_t w) { return __ldg(&t[J][byte_of<K>(w)]); }

template <int K>
__device__ __forceinline__ uint32_t gs(const uint32_t (&t)[256], uint32_t w) { return __ldg(&t[byte_of<K>(w)]); }

// One middle round, the same row choices as tt_round (encryption: row i of column c + i;
// decryption: row i of column c - i).
template <int DIR>
__device__ __forceinline__ void g_round(uint32_t& s0, uint32_t& s1, uint32_t& s2, uint32_t& s3, uint32_t k0, uint32_t k1,
                                        uint32_t k2, uint32_t k3) {
  const uint32_t(&T)[4][256] = DIR == AES_ENCRYPT ? g_small.te : g_small.td;
  uint32_t t0, t1, t2, t3;
  if constexpr (DIR == AES_ENCRYPT) {
    t0 = gl<0, 0>(T, s0) ^ gl<1, 1>(T, s1) ^ gl<2, 2>(T, s2) ^ gl<3, 3>(T, s3) ^ k0;
    t1 = gl<0, 0>(T, s1) ^ gl<1, 1>(T, s2) ^ gl<2, 2>(T, s3) ^ gl<3, 3>(T, s0) ^ k1;
    t2 = gl<0, 0>(T, s2) ^ gl<1, 1>(T, s3) ^ gl<2, 2>(T, s0) ^ gl<3, 3>(T, s1) ^ k2;
    t3 = gl<0, 0>(T, s3) ^ gl<1, 1>(T, s0) ^ gl<2, 2>(T, s1) ^ gl<3, 3>(T, s2) ^ k3;
  } else {
    t0 = gl<0, 0>(T, s0) ^ gl<1, 1>(T, s3) ^ gl<2, 2>(T, s2) ^ gl<3, 3>(T, s1) ^ k0;
    t1 = gl<0, 0>(T, s1) ^ gl<1, 1>(T, s0) ^ gl<2, 2>(T, s3) ^ gl<3, 3>(T, s2) ^ k1;
    t2 = gl<0, 0>(T, s2) ^ gl<1, 1>(T, s1) ^ gl<2, 2>(T, s0) ^ gl<3, 3>(T, s3) ^ k2;
    t3 = gl<0, 0>(T, s3) ^ gl<1, 1>(T, s2) ^ gl<2, 2>(T, s1) ^ gl<3, 3>(T, s0) ^ k3;
  }
  s0 = t0; s1 = t1; s2 = t2; s3 = t3;
}

// Last round (no MixColumns): byte r of output column c is S of row r of column c + r
// (encryption) or c - r (decryption), taken from the S-box word at that byte position.
template <int DIR>
__device__ __forceinline__ uint4 g_final(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3, uint32_t k0, uint32_t k1,
                                         uint32_t k2, uint32_t k3) {
  const uint32_t(&S)[256] = DIR == AES_ENCRYPT ? g_small.s4 : g_small.is4;
  auto col = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return (gs<0>(S, a) & 0x000000FFu) | (gs<1>(S, b) & 0x0000FF00u) | (gs<2>(S, c) & 0x00FF0000u) |
           (gs<3>(S, d) & 0xFF000000u);
  };
  uint4 o;
  if constexpr (DIR == AES_ENCRYPT) {
    o.x = col(s0, s1, s2, s3) ^ k0;
    o.y = col(s1, s2, s3, s0) ^ k1;
    o.z = col(s2, s3, s0, s1) ^ k2;
    o.w = col(s3, s0, s1, s2) ^ k3;
  } else {
    o.x = col(s0, s3, s2, s1) ^ k0;
    o.y = col(s1, s0, s3, s2) ^ k1;
    o.z = col(s2, s1, s0, s3) ^ k2;
    o.w = col(s3, s2, s1, s0) ^ k3;
  }
  return o;
}

constexpr int kSmallThreads = 128;

template <int NR, int DIR>
__global__ void __launch_bounds__(kSmallThreads) tt_small_kernel(const uint4* in, uint4* out, size_t nblocks,
                                                                  const KeyWords kw) {
  const size_t stride = size_t(gridDim.x) * kSmallThreads;
  for (size_t i = size_t(blockIdx.x) * kSmallThreads + threadIdx.x; i < nblocks; i += stride) {
    const uint4 v = tt::ld_block(in + i);
    uint32_t s0 = v.x ^ kw.w[0][0], s1 = v.y ^ kw.w[0][1], s2 = v.z ^ kw.w[0][2], s3 = v.w ^ kw.w[0][3];
#pragma unroll
    for (int r = 1; r < NR; ++r) g_round<DIR>(s0, s1, s2, s3, kw.w[r][0], kw.w[r][1], kw.w[r][2], kw.w[r][3]);
    tt::st_block(out + i, g_final<DIR>(s0, s1, s2, s3, kw.w[NR][0], kw.w[NR][1], kw.w[NR][2], kw.w[NR][3]));
  }
}

// One block with the round keys read from a pool entry (rows in round order, nr of them
// after the first; the same words the batched kernel keeps in registers), the tables from
// global memory.
template <int DIR>
__device__ __forceinline__ uint4 crypt_pool_rows(uint4 v, const uint4* kp, int nr) {
  uint4 k = __ldg(kp);
  uint32_t s0 = v.x ^ k.x, s1 = v.y ^ k.y, s2 = v.z ^ k.z, s3 = v.w ^ k.w;
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    k = __ldg(kp + r);
    g_round<DIR>(s0, s1, s2, s3, k.x, k.y, k.z, k.w);
  }
  for (int r = 10; r < nr; ++r) {  // AES-192 and AES-256: two or four more rounds
    k = __ldg(kp + r);
    g_round<DIR>(s0, s1, s2, s3, k.x, k.y, k.z, k.w);
  }
  k = __ldg(kp + nr);
  return g_final<DIR>(s0, s1, s2, s3, k.x, k.y, k.z, k.w);
}

// Every block of the batch's messages (at most kSmallBatchMax, both directions, any key size)
// in one grid-stride loop: a thread finds its block's message by a scan of the starts in the
// constant bank.
__global__ void __launch_bounds__(kSmallThreads) small_batch_kernel(const __grid_constant__ SmallBatch b,
                                                                     const PoolEntry* pool) {
  const uint64_t total = b.start[b.n];
  const uint64_t stride = uint64_t(gridDim.x) * kSmallThreads;
  for (uint64_t g = uint64_t(blockIdx.x) * kSmallThreads + threadIdx.x; g < total; g += stride) {
    uint32_t m = 0;
    while (g >= b.start[m + 1]) ++m;
    const SmallMsg& d = b.m[m];
    const uint64_t j = g - b.start[m];
    const PoolEntry* e = pool + d.key_idx;
    const int nr = __ldg(&e->nr);
    const uint4 v = tt::ld_block(reinterpret_cast<const uint4*>(d.src) + j);
    const uint4 o = d.dir == AES_ENCRYPT ? crypt_pool_rows<AES_ENCRYPT>(v, reinterpret_cast<const uint4*>(e->enc), nr)
                                         : crypt_pool_rows<AES_DECRYPT>(v, reinterpret_cast<const uint4*>(e->dec), nr);
    tt::st_block(reinterpret_cast<uint4*>(d.dst) + j, o);
  }
}

using SmallFn = void (*)(const uint4*, uint4*, size_t, const KeyWords);

SmallFn pick_small(int dir, int nr) {
  if (dir == AES_ENCRYPT)
    return nr == 10 ? tt_small_kernel<10, AES_ENCRYPT> : nr == 12 ? tt_small_kernel<12, AES_ENCRYPT>
                                                                  : tt_small_kernel<14, AES_ENCRYPT>;
  return nr == 10 ? tt_small_kernel<10, AES_DECRYPT> : nr == 12 ? tt_small_kernel<12, AES_DECRYPT>
                                                                : tt_small_kernel<14, AES_DECRYPT>;
}

}  // namespace

aes_status launch_small(int dir, int nr, const KeyWords& kw, const void* d_in, void* d_out, size_t nblocks,
                        cudaStream_t stream) {
  if (nr != 10 && nr != 12 && nr != 14) return set_error(AES_EINVAL, "no small-call kernel for nr=%d", nr);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  const size_t want = (nblocks + kSmallThreads - 1) / kSmallThreads;
  const size_t cap = size_t(di->sms) * 16;  // a grid-stride loop beyond 16 CTAs per SM
  const unsigned grid = unsigned(want < cap ? want : cap);
  pick_small(dir, nr)<<<grid, kSmallThreads, 0, stream>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                                         nblocks, kw);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "small-call kernel launch");
  return AES_OK;
}

aes_status launch_small_batch(const SmallBatch& b, const PoolEntry* pool, cudaStream_t stream) {
  if (b.n == 0 || b.n > uint32_t(kSmallBatchMax)) return set_error(AES_EINVAL, "small batch of %u messages", b.n);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  const uint64_t total = b.start[b.n];
  if (total == 0) return AES_OK;
  const uint64_t want = (total + kSmallThreads - 1) / kSmallThreads;
  const uint64_t cap = uint64_t(di->sms) * 16;
  small_batch_kernel<<<unsigned(want < cap ? want : cap), kSmallThreads, 0, stream>>>(b, pool);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "small-batch kernel launch");
  return AES_OK;
}

}  // namespace aesgb
