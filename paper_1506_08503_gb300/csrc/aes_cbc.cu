// aes_cbc.cu -- the paper's CBC mode over whole messages (Section II; App. A1 encryption,
// App. A4 decryption): an N x M byte matrix of N messages with M bytes each, one IV per message
// (or one IV for all, as the appendix does with a repeated IV), C_j = E(P_j ^ C_{j-1}) with
// C_{-1} = IV, and P_j = D(C_j) ^ C_{j-1}.
//
// Encryption is a chain inside each message, so it runs one lane per message: the lane walks
// its row block by block, keeping the chaining value in registers.  With few messages the
// chain's latency is the bound; the direct kernel then spreads the lanes over all SMs and
// loads each lane's next block itself.  With enough messages to fill the GPU (78K or more)
// the tiled kernel moves rows through shared memory so that every global access is coalesced,
// and the shared-memory lookups are the bound, as for independent blocks.
//
// Decryption has no chain: every block needs only its own ciphertext and the previous one, so
// it runs one block per lane over the whole matrix like the independent-block kernel, with
// one extra (mostly L1-hit) load of the previous block.  It cannot run in place.
#include <algorithm>

#include "aes_ttable.cuh"
#include "aesgb_testing.h"

namespace aesgb {
namespace {

using namespace tt;

__device__ __forceinline__ uint4 ld_cached(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
  return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// IVs: iv_stride 0 = one IV (16 bytes at ivs) for every message, 1 = one IV per message.
template <int NR>
__global__ void __launch_bounds__(512, 1)
cbc_encrypt_kernel(const uint4* in, uint4* out, const uint4* ivs, int iv_stride, uint64_t nmsgs, uint64_t mblocks,
                   const KeyWords kw) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lc = (threadIdx.x & 31u) * 4u;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t msg = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; msg < nmsgs; msg += stride) {
    const uint4* src = in + msg * mblocks;
    uint4* dst = out + msg * mblocks;
    uint4 chain = ld_cached(ivs + (iv_stride ? msg : 0));
    uint4 next = mblocks ? ld_cached(src) : make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t j = 0; j < mblocks; ++j) {
      const uint4 p = next;
      if (j + 1 < mblocks) next = ld_cached(src + j + 1);
      chain = crypt_block<NR, AES_ENCRYPT>(xor4(p, chain), kw, sm, lc);
      st_block(dst + j, chain);
    }
  }
}

// Few messages: the chain's latency is the bound.  One lane per chain spends it issuing a
// whole block's round (16 byte permutes and lookups) before the next round can start; here
// four lanes share a chain, lane q holding column q of the state (col_round: four lookups,
// three shuffles, two XORs per lane and round).  A warp runs `cpw` chains (lanes 4 cpw.. idle)
// and the first `wpc` warps of a CTA run chains (all of them fill the tables): with few chains
// one per warp, since every chain a warp adds makes each of its shuffles and lookups slower;
// with many, up to eight per warp, since the SM's shared-memory pipe is then the bound.  Each
// lane keeps its column of every round key in registers; the four lanes of a chain load and
// store one 16-byte block together.  The next block's plaintext, the first round key and the
// last one are combined off the chain's dependent path.
constexpr unsigned kColMaxThreads = 256;
constexpr uint64_t kColChainsPerSm = 64;  // up to 8 warps of 8 chains per SM

template <int NR>
__global__ void __launch_bounds__(kColMaxThreads, 1)
cbc_encrypt_cols(const uint4* in, uint4* out, const uint4* ivs, int iv_stride, uint64_t nmsgs, uint64_t mblocks,
                 const KeyWords kw, uint32_t cpw, uint32_t wpc) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lane = threadIdx.x & 31u, q = lane & 3u, slot = lane >> 2;
  const uint32_t lc = lane * 4u;
  if (slot >= cpw || (threadIdx.x >> 5) >= wpc) return;
  uint32_t kq[NR + 1];
#pragma unroll
  for (int r = 0; r <= NR; ++r) kq[r] = kw.w[r][q];
  const uint32_t k_last_first = kq[NR] ^ kq[0];
  // warp w of CTA b is global warp w * grid + b: consecutive chains go to different SMs first
  const uint64_t warp = uint64_t(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint64_t step = uint64_t(gridDim.x) * wpc * cpw;
  for (uint64_t msg = warp * cpw + slot; msg < nmsgs; msg += step) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(in + msg * mblocks) + q;
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + msg * mblocks) + q;
    // coherent loads: encryption may run in place
    uint32_t s = src[0] ^ reinterpret_cast<const uint32_t*>(ivs + (iv_stride ? msg : 0))[q] ^ kq[0];
    for (uint64_t j = 0; j < mblocks; ++j) {
      const uint32_t next = j + 1 < mblocks ? src[4 * (j + 1)] : 0u;
#pragma unroll
      for (int r = 1; r < NR; ++r) s = col_round(s, kq[r], sm, lane, lc);
      const uint32_t p = col_last(s, sm, lane, lc);
      dst[4 * j] = p ^ kq[NR];
      s = p ^ (next ^ k_last_first);  // C_j ^ P_j+1 ^ K_0
    }
  }
}

// Many messages: each warp owns kRows = 32 consecutive messages (one chain per lane) and
// moves them through shared memory kStage blocks at a time, so that global loads and stores
// are coalesced (a warp instruction covers 4 rows x 128 contiguous bytes instead of 32
// scattered rows, whose separate cache lines would cost L1 cycles the T-table lookups need).
// Tile rows are padded to kStage + 1 entries, which puts the 8 lanes of each quarter-warp in
// different bank groups both when a lane walks its own row and when the warp copies the tile.
// The next stage is loaded into registers while the current one is enciphered.  (Two chains
// per lane, in lockstep over a 64-row tile, measured slower: 572 against 625 GB/s.)
constexpr int kStage = 8;
constexpr uint32_t kRows = 32;
constexpr uint32_t kTileBytes = kRows * (kStage + 1) * 16u;  // per warp
constexpr uint32_t kStagedThreads = 640;  // the largest CTA whose tiles fit beside the tables
constexpr int kPer = int(kRows) * kStage / 32;  // tile elements per lane

template <int NR, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
cbc_encrypt_staged(const uint4* in, uint4* out, const uint4* ivs, int iv_stride, uint64_t nmsgs, uint64_t mblocks,
                   const KeyWords kw) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t lc = lane * 4u;
  uint4* tile = reinterpret_cast<uint4*>(reinterpret_cast<char*>(smem) + 2u * kRegion + warp * kTileBytes);
  const uint64_t ngroups = (nmsgs + kRows - 1) / kRows;
  const uint64_t nw = uint64_t(gridDim.x) * (THREADS / 32);
  for (uint64_t grp = uint64_t(blockIdx.x) * (THREADS / 32) + warp; grp < ngroups; grp += nw) {
    const uint64_t m0 = grp * kRows;
    const uint32_t rows = uint32_t(nmsgs - m0 < kRows ? nmsgs - m0 : kRows);
    uint4 chain = lane < rows ? ld_cached(ivs + (iv_stride ? m0 + lane : 0)) : make_uint4(0u, 0u, 0u, 0u);
    // element e = i * 32 + lane of a stage is block (e mod kStage) of row (e / kStage)
    uint4 pre[kPer];
    auto load_stage = [&](uint64_t j0) {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t e = uint32_t(i) * 32u + lane, r = e / kStage, b = e % kStage;
        pre[i] = (r < rows && j0 + b < mblocks) ? ld_block(in + (m0 + r) * mblocks + j0 + b) : make_uint4(0u, 0u, 0u, 0u);
      }
    };
    load_stage(0);
    for (uint64_t j0 = 0; j0 < mblocks; j0 += kStage) {
      const uint32_t sb = uint32_t(mblocks - j0 < kStage ? mblocks - j0 : kStage);
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t e = uint32_t(i) * 32u + lane, r = e / kStage, b = e % kStage;
        if (r < rows && b < sb) tile[r * (kStage + 1) + b] = pre[i];
      }
      __syncwarp();
      if (j0 + kStage < mblocks) load_stage(j0 + kStage);
      if (lane < rows) {
        uint4* row = tile + lane * (kStage + 1);
        for (uint32_t b = 0; b < sb; ++b) {
          chain = crypt_block<NR, AES_ENCRYPT>(xor4(row[b], chain), kw, sm, lc);
          row[b] = chain;
        }
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t e = uint32_t(i) * 32u + lane, r = e / kStage, b = e % kStage;
        if (r < rows && b < sb) st_block(out + (m0 + r) * mblocks + j0 + b, tile[r * (kStage + 1) + b]);
      }
      __syncwarp();  // the tile is rewritten by the next stage
    }
  }
}

// Decryption, one lane per block in grid-stride order.  The block's message and position in
// it advance with the stride (its quotient and remainder by the message length come from the
// host), so no lane divides per block.
constexpr unsigned kDecThreads = 768;  // 24 warps per SM, as in the tuned independent-block kernel

template <int NR>
__global__ void __launch_bounds__(kDecThreads, 1)
cbc_decrypt_kernel(const uint4* in, uint4* out, const uint4* ivs, int iv_stride, uint64_t nmsgs, uint64_t mblocks,
                   const KeyWords kw, uint64_t stride_q, uint64_t stride_r) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_DECRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lc = (threadIdx.x & 31u) * 4u;
  const uint64_t total = nmsgs * mblocks;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  uint64_t msg = g / mblocks, j = g - msg * mblocks;  // once per thread
  auto advance = [&](uint64_t& m, uint64_t& q) {
    m += stride_q;
    q += stride_r;
    if (q >= mblocks) {
      q -= mblocks;
      ++m;
    }
  };
  // two blocks in flight per thread (g and g + stride), as in the independent-block kernel
  for (; g + stride < total; g += 2 * stride) {
    uint64_t msg1 = msg, j1 = j;
    advance(msg1, j1);
    const uint4 c0 = ld_cached(in + g), c1 = ld_cached(in + g + stride);
    const uint4 p0 = j ? ld_cached(in + g - 1) : ld_cached(ivs + (iv_stride ? msg : 0));
    const uint4 p1 = j1 ? ld_cached(in + g + stride - 1) : ld_cached(ivs + (iv_stride ? msg1 : 0));
    const uint4 d0 = crypt_block<NR, AES_DECRYPT>(c0, kw, sm, lc);
    const uint4 d1 = crypt_block<NR, AES_DECRYPT>(c1, kw, sm, lc);
    st_block(out + g, xor4(d0, p0));
    st_block(out + g + stride, xor4(d1, p1));
    msg = msg1;
    j = j1;
    advance(msg, j);
  }
  if (g < total) {
    const uint4 c = ld_cached(in + g);
    const uint4 prev = j ? ld_cached(in + g - 1) : ld_cached(ivs + (iv_stride ? msg : 0));
    st_block(out + g, xor4(crypt_block<NR, AES_DECRYPT>(c, kw, sm, lc), prev));
  }
}

using CbcKernel = void (*)(const uint4*, uint4*, const uint4*, int, uint64_t, uint64_t, const KeyWords);
using CbcDecKernel = void (*)(const uint4*, uint4*, const uint4*, int, uint64_t, uint64_t, const KeyWords, uint64_t,
                              uint64_t);

template <int THREADS>
CbcKernel pick_staged_nr(int nr) {
  return nr == 10 ? cbc_encrypt_staged<10, THREADS>
                  : nr == 12 ? cbc_encrypt_staged<12, THREADS> : cbc_encrypt_staged<14, THREADS>;
}

// CTA size of the staged kernel.  Its warps (one CTA per SM) take the 32-message groups in
// waves, and every chain of a group is as long as the others, so the last wave, if partly
// filled, costs a whole wave.  Of 16, 18 and 20 warps per CTA the size with the fewest waves
// wins, the smaller one among equals (fewer warps finish a wave no later).  2^18 messages on
// 152 SMs: 16 warps take 4 waves, 18 warps 3 (all but full), 20 warps 3 (the last 69 % full).
unsigned staged_threads(uint64_t ngroups, int sms) {
  unsigned best = kStagedThreads;
  uint64_t best_waves = UINT64_MAX;
  for (unsigned t = 512; t <= kStagedThreads; t += 64) {
    const uint64_t per_wave = uint64_t(sms) * (t / 32);
    const uint64_t waves = (ngroups + per_wave - 1) / per_wave;
    if (waves < best_waves) {
      best_waves = waves;
      best = t;
    }
  }
  return best;
}

CbcKernel pick_staged(int nr, unsigned threads) {
  return threads == 512 ? pick_staged_nr<512>(nr) : threads == 576 ? pick_staged_nr<576>(nr) : pick_staged_nr<640>(nr);
}

using CbcColsKernel = void (*)(const uint4*, uint4*, const uint4*, int, uint64_t, uint64_t, const KeyWords, uint32_t,
                              uint32_t);

CbcColsKernel pick_cols(int nr) {
  return nr == 10 ? cbc_encrypt_cols<10> : nr == 12 ? cbc_encrypt_cols<12> : cbc_encrypt_cols<14>;
}

CbcKernel pick_encrypt(int nr) {
  return nr == 10 ? cbc_encrypt_kernel<10> : nr == 12 ? cbc_encrypt_kernel<12> : cbc_encrypt_kernel<14>;
}

CbcDecKernel pick_decrypt(int nr) {
  return nr == 10 ? cbc_decrypt_kernel<10> : nr == 12 ? cbc_decrypt_kernel<12> : cbc_decrypt_kernel<14>;
}

}  // namespace

ColsShape cols_shape(uint64_t chains, int sms) {
  const uint64_t per_sm = (chains + uint64_t(sms) - 1) / uint64_t(sms);
  unsigned warps, cpw;
  if (per_sm <= 4) {  // latency-bound: one chain per warp, at most one warp per scheduler
    cpw = 1;
    warps = unsigned(per_sm);
  } else if (per_sm <= 32) {  // four warps, the chains shared out among them
    warps = 4;
    cpw = unsigned((per_sm + 3) / 4);
  } else {  // the shared-memory pipe is the bound: eight chains per warp
    cpw = 8;
    warps = unsigned(std::min<uint64_t>(kColMaxThreads / 32, (per_sm + 7) / 8));
  }
  const uint64_t per_cta = uint64_t(warps) * cpw;
  const uint64_t want = (chains + per_cta - 1) / per_cta;
  return ColsShape{std::max(128u, 32u * warps), warps, unsigned(std::min<uint64_t>(want, uint64_t(sms))), cpw};
}

}  // namespace aesgb

using namespace aesgb;

extern "C" int aes_testing_cols_shape(uint64_t chains, int sms, unsigned* threads, unsigned* wpc, unsigned* grid,
                                      unsigned* cpw) {
  if (chains == 0 || sms < 1 || !threads || !wpc || !grid || !cpw) return -1;
  const ColsShape sh = cols_shape(chains, sms);
  *threads = sh.threads;
  *wpc = sh.wpc;
  *grid = sh.grid;
  *cpw = sh.cpw;
  return 0;
}

extern "C" aes_status aes_cbc_crypt(const aes_key_schedule* ks, const void* d_ivs, int iv_per_msg, const void* d_in,
                                    void* d_out, size_t nmsgs, size_t blocks_per_msg, int dir, void* cuda_stream) {
  clear_error();
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (iv_per_msg != 0 && iv_per_msg != 1) return set_error(AES_EINVAL, "iv_per_msg must be 0 or 1");
  if (nmsgs == 0 || blocks_per_msg == 0) return AES_OK;
  if (!d_in || !d_out || !d_ivs) return set_error(AES_EINVAL, "null buffer");
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out) | reinterpret_cast<uintptr_t>(d_ivs)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  if (blocks_per_msg > (SIZE_MAX >> 5) / nmsgs) return set_error(AES_EINVAL, "matrix too large");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  const uintptr_t bytes = uintptr_t(nmsgs) * blocks_per_msg * 16u;
  if (a != b && a < b + bytes && b < a + bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  if (dir == AES_DECRYPT && a == b)
    return set_error(AES_EINVAL, "CBC decryption cannot run in place (each block needs the previous ciphertext)");
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  // the kernel adds the IV itself: the schedule goes in without one
  const KeyWords kw = dir == AES_ENCRYPT ? enc_key_words(*ks, nullptr) : dec_key_words(*ks, nullptr);
  // encryption of enough messages to give every warp of a full GPU 32 of them takes the
  // staged kernel; fewer messages are latency-bound chains, better spread one per lane
  const bool staged = dir == AES_ENCRYPT && nmsgs >= uint64_t(di->sms) * kStagedThreads;
  const unsigned staged_cta = staged ? staged_threads((nmsgs + kRows - 1) / kRows, di->sms) : 0u;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  // few chains: four lanes per chain
  if (dir == AES_ENCRYPT && !staged && nmsgs <= uint64_t(di->sms) * kColChainsPerSm) {
    const CbcColsKernel kc = pick_cols(ks->nr);
    const size_t smem = ttable_smem_bytes(dir);
    aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(kc), smem);
    if (ast != AES_OK) return ast;
    const ColsShape sh = cols_shape(nmsgs, di->sms);
    kc<<<sh.grid, sh.threads, smem, st>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                          static_cast<const uint4*>(d_ivs), iv_per_msg, nmsgs, blocks_per_msg, kw, sh.cpw,
                                          sh.wpc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CBC kernel launch");
    return AES_OK;
  }
  CbcKernel k = dir == AES_DECRYPT ? nullptr
                : staged           ? pick_staged(ks->nr, staged_cta)
                                   : pick_encrypt(ks->nr);
  CbcDecKernel kd = dir == AES_DECRYPT ? pick_decrypt(ks->nr) : nullptr;
  const size_t smem = ttable_smem_bytes(dir) + (staged ? size_t(staged_cta / 32) * kTileBytes : 0);
  aes_status ast = ensure_kernel_smem(k ? reinterpret_cast<const void*>(k) : reinterpret_cast<const void*>(kd), smem);
  if (ast != AES_OK) return ast;
  unsigned threads = dir == AES_DECRYPT ? kDecThreads : 512u;
  uint64_t work = uint64_t(nmsgs) * blocks_per_msg;
  if (staged) {
    threads = staged_cta;  // the kernel instance's warp-to-group map assumes this CTA size
    work = (nmsgs + kRows - 1) / kRows * 32;  // kRows messages per warp
  } else if (dir == AES_ENCRYPT) {
    // a lane per message: with few messages, spread the chains over all SMs (smaller CTAs)
    // rather than packing them into a few
    work = nmsgs;
    const uint64_t per_sm = (work + di->sms - 1) / di->sms;
    threads = per_sm >= 512 ? 512u : unsigned(((per_sm + 31) / 32) * 32);
  }
  const uint64_t want = (work + threads - 1) / threads;
  const unsigned grid = unsigned(want < uint64_t(di->sms) ? want : uint64_t(di->sms));
  if (kd) {
    const uint64_t stride = uint64_t(grid) * threads;
    kd<<<grid, threads, smem, st>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                    static_cast<const uint4*>(d_ivs), iv_per_msg, nmsgs, blocks_per_msg, kw,
                                    stride / blocks_per_msg, stride % blocks_per_msg);
  } else {
    k<<<grid, threads, smem, st>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                   static_cast<const uint4*>(d_ivs), iv_per_msg, nmsgs, blocks_per_msg, kw);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CBC kernel launch");
  return AES_OK;
}
