// aes_cbc_batched.cu -- the paper's CBC mode over many messages of different lengths, each with
// its own key (a key-pool slot: the key tensor K of Section II) and its own IV (a row of the IV
// matrix V): C_j = E_Ki(P_j ^ C_{j-1}), C_{-1} = IV_i (App. A1), and P_j = D_Ki(C_j) ^ C_{j-1}
// (App. A4).
//
// Encryption is a chain inside each message.  Up to 64 messages per SM run four lanes to a
// message (a lane per state column, as aes_cbc_crypt does with few messages), more run one
// lane per message; the host sorts the messages by length (longest first), so that the chains
// sharing a warp finish together, and the round keys stay in registers (AES-128/192/256
// mixed: the round count is read with the key).  Its rate is the chain's latency, one block
// per ten to fourteen dependent rounds per message.
//
// Decryption has no chain: it is the batched kernel (messages laid end to end, warp slices of
// equal work in blocks x rounds) with each block's output XORed with the previous ciphertext
// block of its message, or with the message's IV for the first block.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "aes_batched.cuh"

namespace aesgb {
namespace {

using namespace tt;

struct CbcMsg {
  uint64_t src_block, dst_block, nblocks;
  uint32_t key_idx, pad;
  uint4 iv;
};
static_assert(sizeof(CbcMsg) == 48, "CBC message descriptors are 48 bytes");

constexpr int kEncMaxThreads = 512;

__global__ void __launch_bounds__(kEncMaxThreads, 1)
cbc_enc_msgs(uint64_t in_base, uint64_t out_base, const CbcMsg* msgs, uint32_t n, const PoolEntry* pool) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lc = (threadIdx.x & 31u) * 4u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += stride) {
    const CbcMsg* d = msgs + m;
    const uint64_t nb = ldg64(&d->nblocks);
    const uint4* src = reinterpret_cast<const uint4*>(in_base + ldg64(&d->src_block) * 16u);
    uint4* dst = reinterpret_cast<uint4*>(out_base + ldg64(&d->dst_block) * 16u);
    uint32_t kw[kMaxRounds + 1][4], kl[4];
    int nr;
    load_key<AES_ENCRYPT>(pool, __ldg(&d->key_idx), kw, kl, nr);
    uint4 chain = __ldg(&d->iv);
    uint4 next = nb ? __ldg(src) : make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t j = 0; j < nb; ++j) {
      const uint4 p = next;
      if (j + 1 < nb) next = __ldg(src + j + 1);
      chain = crypt_rt<AES_ENCRYPT>(xor4(p, chain), kw, kl, nr, sm, lc);
      st_block(dst + j, chain);
    }
  }
}

// Few messages: four lanes per message (tt::col_round), lane q holding column q of the state
// and of every round key, `cpw` messages per warp in the first `wpc` warps of each CTA (see
// cols_shape); consecutive messages (the longest first) go to different SMs first.
constexpr int kColMaxThreads = 256;
constexpr uint64_t kColChainsPerSm = 64;

__global__ void __launch_bounds__(kColMaxThreads, 1)
cbc_enc_msgs_cols(uint64_t in_base, uint64_t out_base, const CbcMsg* msgs, uint32_t n, const PoolEntry* pool,
                  uint32_t cpw, uint32_t wpc) {
  extern __shared__ __align__(16) uint32_t smem[];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lane = threadIdx.x & 31u, q = lane & 3u, slot = lane >> 2;
  const uint32_t lc = lane * 4u;
  if (slot >= cpw || (threadIdx.x >> 5) >= wpc) return;
  const uint32_t warp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint32_t step = gridDim.x * wpc * cpw;
  for (uint32_t m = warp * cpw + slot; m < n; m += step) {
    const CbcMsg* d = msgs + m;
    const uint64_t nb = ldg64(&d->nblocks);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(in_base + ldg64(&d->src_block) * 16u) + q;
    uint32_t* dst = reinterpret_cast<uint32_t*>(out_base + ldg64(&d->dst_block) * 16u) + q;
    const PoolEntry* e = pool + __ldg(&d->key_idx);
    const int nr = __ldg(&e->nr);
    uint32_t kq[kMaxRounds];
#pragma unroll
    for (int r = 0; r < kMaxRounds; ++r) kq[r] = __ldg(&e->enc[r][q]);
    const uint32_t kl = __ldg(&e->enc[nr][q]);
    const uint32_t k_last_first = kl ^ kq[0];
    // coherent loads of the data: encryption may run in place
    uint32_t s = nb ? src[0] ^ __ldg(reinterpret_cast<const uint32_t*>(&d->iv) + q) ^ kq[0] : 0u;
    for (uint64_t j = 0; j < nb; ++j) {
      const uint32_t next = j + 1 < nb ? src[4 * (j + 1)] : 0u;
#pragma unroll
      for (int r = 1; r < 10; ++r) s = col_round(s, kq[r], sm, lane, lc);
      if (nr > 10) {  // the same in the four lanes of a message
        s = col_round(s, kq[10], sm, lane, lc);
        s = col_round(s, kq[11], sm, lane, lc);
        if (nr > 12) {
          s = col_round(s, kq[12], sm, lane, lc);
          s = col_round(s, kq[13], sm, lane, lc);
        }
      }
      const uint32_t p = col_last(s, sm, lane, lc);
      dst[4 * j] = p ^ kl;
      s = p ^ (next ^ k_last_first);  // C_j ^ P_j+1 ^ K_0
    }
  }
}

constexpr int kDecThreads = 512, kDecU = 2;

__global__ void __launch_bounds__(kDecThreads, 1)
cbc_dec_msgs(uint64_t in_base, uint64_t out_base, const BatchDir bd, const PoolEntry* pool) {
  extern __shared__ __align__(16) uint32_t smem[];
  batched_body<AES_DECRYPT, kDecThreads, kDecU, 0, true>(in_base, out_base, bd, pool, blockIdx.x, gridDim.x, smem);
}

// Buffers kept in the pool between calls: pinned staging and its device copy, and an event
// marking the end of the last call's kernels (which read the device copy).
struct CbcCtx {
  int device = -1;
  size_t cap = 0;
  uint8_t* host = nullptr;
  uint8_t* dev = nullptr;
  cudaEvent_t used = nullptr;
};

void free_ctx(CbcCtx* c) {
  if (!c) return;
  if (c->used) { cudaEventSynchronize(c->used); cudaEventDestroy(c->used); }
  if (c->dev) cudaFree(c->dev);
  if (c->host) cudaFreeHost(c->host);
  delete c;
}

aes_status ensure_ctx(aes_keypool* pool, size_t bytes, CbcCtx** out) {
  CbcCtx* c = static_cast<CbcCtx*>(pool->cbc);
  if (c && c->cap >= bytes) {
    *out = c;
    return AES_OK;
  }
  free_ctx(c);
  pool->cbc = nullptr;
  c = new CbcCtx();
  c->device = pool->device;
  c->cap = std::max<size_t>(bytes, size_t(1) << 20);
  cudaError_t e;
  if ((e = cudaMallocHost(&c->host, c->cap)) != cudaSuccess || (e = cudaMalloc(&c->dev, c->cap)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->used, cudaEventDisableTiming)) != cudaSuccess) {
    free_ctx(c);
    return set_error(AES_ENOMEM, "CBC descriptor buffers (%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  pool->cbc = c;
  *out = c;
  return AES_OK;
}

size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

}  // namespace

void cbc_batched_release(aes_keypool* pool) {
  if (!pool) return;
  free_ctx(static_cast<CbcCtx*>(pool->cbc));
  pool->cbc = nullptr;
}

}  // namespace aesgb

using namespace aesgb;

extern "C" aes_status aes_cbc_batched(aes_keypool* pool, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs,
                                      const void* d_in, void* d_out, size_t buf_bytes, void* cuda_stream) {
  clear_error();
  if (!pool || !pool->entries || !pool->mu) return set_error(AES_EINVAL, "null key pool");
  if (nmsgs && !msgs) return set_error(AES_EINVAL, "null message array");
  if (nmsgs > (size_t(1) << 24)) return set_error(AES_EINVAL, "%zu messages exceed 2^24", nmsgs);
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), o = reinterpret_cast<uintptr_t>(d_out);
  const bool overlap = a < o + buf_bytes && o < a + buf_bytes;
  if (a != o && overlap) return set_error(AES_EINVAL, "input and output overlap without being identical");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev != pool->device) return set_error(AES_EINVAL, "pool belongs to device %d, current device is %d", pool->device, dev);
  std::vector<size_t> enc, dec;
  for (size_t i = 0; i < nmsgs; ++i) {
    const aes_msg& m = msgs[i];
    if (m.dir != AES_ENCRYPT && m.dir != AES_DECRYPT) return set_error(AES_EINVAL, "message %zu: bad dir %u", i, m.dir);
    if ((m.offset | m.length) & 15u) return set_error(AES_EINVAL, "message %zu: offset and length must be multiples of 16", i);
    if (m.offset > buf_bytes || m.length > buf_bytes - m.offset)
      return set_error(AES_EINVAL, "message %zu leaves the %zu-byte buffers", i, buf_bytes);
    if (m.length == 0) continue;
    if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
    if (size_t(m.key_idx) >= pool->capacity || pool->nr[m.key_idx] == 0)
      return set_error(AES_EINVAL, "message %zu: key slot %u is not loaded", i, m.key_idx);
    (m.dir == AES_ENCRYPT ? enc : dec).push_back(i);
  }
  if (!dec.empty() && overlap)
    return set_error(AES_EINVAL, "CBC decryption cannot run in place (each block needs the previous ciphertext)");
  if (enc.empty() && dec.empty()) return AES_OK;
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(pool->mu));

  // decryption grid: one CTA per SM, fewer when there is less than a block per thread
  uint64_t td = 0;
  for (size_t k : dec) td += msgs[k].length / 16;
  const uint64_t dgrid = dec.empty() ? 0 : std::max<uint64_t>(1, std::min<uint64_t>(di->sms, (td + kDecThreads - 1) / kDecThreads));
  // layout: encryption descriptors | decryption descriptors | starts | warp slices | IVs
  const size_t nw = size_t(dgrid) * (kDecThreads / 32);
  const size_t off_enc = 0, off_dmsg = align16(enc.size() * sizeof(CbcMsg));
  const size_t off_start = align16(off_dmsg + dec.size() * sizeof(BatchMsg));
  const size_t off_gb = align16(off_start + (dec.size() + 1) * sizeof(uint64_t));
  const size_t off_wm = align16(off_gb + (nw + 1) * sizeof(uint64_t));
  const size_t off_iv = align16(off_wm + nw * sizeof(uint32_t));
  const size_t total = off_iv + dec.size() * 16;
  CbcCtx* c = nullptr;
  aes_status st = ensure_ctx(pool, total, &c);
  if (st != AES_OK) return st;
  if ((e = cudaEventSynchronize(c->used)) != cudaSuccess) return cuda_error(e, "waiting for the previous call");
  uint8_t* h = c->host;
  // encryption: longest messages first, so that the lanes of a warp run chains of similar length
  std::sort(enc.begin(), enc.end(), [&](size_t x, size_t y) { return msgs[x].length > msgs[y].length; });
  CbcMsg* em = reinterpret_cast<CbcMsg*>(h + off_enc);
  for (size_t k = 0; k < enc.size(); ++k) {
    const aes_msg& m = msgs[enc[k]];
    em[k] = CbcMsg{m.offset / 16, m.offset / 16, m.length / 16, m.key_idx, 0u, make_uint4(0u, 0u, 0u, 0u)};
    if (ivs) std::memcpy(&em[k].iv, ivs + 16 * enc[k], 16);
  }
  BatchMsg* dm = reinterpret_cast<BatchMsg*>(h + off_dmsg);
  uint64_t* ds = reinterpret_cast<uint64_t*>(h + off_start);
  uint4* div = reinterpret_cast<uint4*>(h + off_iv);
  uint64_t pos = 0;
  for (size_t k = 0; k < dec.size(); ++k) {
    const aes_msg& m = msgs[dec[k]];
    dm[k] = BatchMsg{m.key_idx, 0u, m.offset / 16, m.offset / 16, m.length / 16};
    ds[k] = pos;
    pos += dm[k].nblocks;
    if (ivs) std::memcpy(div + k, ivs + 16 * dec[k], 16);
    else div[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  ds[dec.size()] = td;
  if (!dec.empty()) {
    weighted_slices(dm, ds, dec.size(), pool->nr, work_of(dm, dec.size(), pool->nr), dgrid * (kDecThreads / 32),
                    reinterpret_cast<uint64_t*>(h + off_gb), reinterpret_cast<uint32_t*>(h + off_wm));
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if ((e = cudaMemcpyAsync(c->dev, h, total, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_error(e, "descriptor upload");
  const uint64_t in_base = reinterpret_cast<uint64_t>(d_in), out_base = reinterpret_cast<uint64_t>(d_out);
  if (!enc.empty() && enc.size() <= uint64_t(di->sms) * kColChainsPerSm) {
    const size_t smem = ttable_smem_bytes(AES_ENCRYPT);
    if ((st = ensure_kernel_smem(reinterpret_cast<const void*>(cbc_enc_msgs_cols), smem)) != AES_OK) return st;
    const ColsShape sh = cols_shape(enc.size(), di->sms);
    cbc_enc_msgs_cols<<<sh.grid, sh.threads, smem, s>>>(in_base, out_base, reinterpret_cast<const CbcMsg*>(c->dev + off_enc),
                                                        uint32_t(enc.size()), pool->entries, sh.cpw, sh.wpc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CBC encryption launch");
  } else if (!enc.empty()) {
    const size_t smem = ttable_smem_bytes(AES_ENCRYPT);
    if ((st = ensure_kernel_smem(reinterpret_cast<const void*>(cbc_enc_msgs), smem)) != AES_OK) return st;
    // a lane per message, spread over the SMs when there are few (the chains are the bound)
    const uint64_t per_sm = (enc.size() + di->sms - 1) / di->sms;
    const unsigned threads = per_sm >= kEncMaxThreads ? unsigned(kEncMaxThreads) : unsigned(((per_sm + 31) / 32) * 32);
    const uint64_t want = (enc.size() + threads - 1) / threads;
    const unsigned grid = unsigned(std::min<uint64_t>(want, di->sms));
    cbc_enc_msgs<<<grid, threads, smem, s>>>(in_base, out_base, reinterpret_cast<const CbcMsg*>(c->dev + off_enc),
                                              uint32_t(enc.size()), pool->entries);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CBC encryption launch");
  }
  if (!dec.empty()) {
    const size_t smem = ttable_smem_bytes(AES_DECRYPT);
    if ((st = ensure_kernel_smem(reinterpret_cast<const void*>(cbc_dec_msgs), smem)) != AES_OK) return st;
    const BatchDir bd{reinterpret_cast<const BatchMsg*>(c->dev + off_dmsg), reinterpret_cast<const uint64_t*>(c->dev + off_start),
                      reinterpret_cast<const uint32_t*>(c->dev + off_wm), td, uint32_t(dec.size()), 0u,
                      reinterpret_cast<const uint64_t*>(c->dev + off_gb), reinterpret_cast<const uint4*>(c->dev + off_iv)};
    cbc_dec_msgs<<<unsigned(dgrid), kDecThreads, smem, s>>>(in_base, out_base, bd, pool->entries);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "CBC decryption launch");
  }
  if ((e = cudaEventRecord(c->used, s)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  return AES_OK;
}
