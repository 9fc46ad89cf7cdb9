// aes_keypool.cu -- device-resident key schedules (the paper's per-message key tensor K,
// Section II) and their expansion on the device.
//
// One thread expands one key: the AES-128 schedule of App. A3 (RotWord + SubWord + Rcon on
// every fourth word, then a running XOR), and for 192/256-bit keys the general Nk-word rule
// of FIPS-197 Section 5.2 (SubWord alone at i = 4 mod 8 when Nk = 8).  The same thread
// also writes the decryption words of the equivalent inverse cipher: K[nr] first,
// InvMixColumns(K[nr - r]) for the middle rounds and K[0] last.
#include <cstring>
#include <mutex>
#include <new>

#include "aes_internal.cuh"

namespace aesgb {
namespace {

static __device__ const FieldTables g_pool_tables = make_field_tables();

constexpr size_t kMaxPool = size_t(1) << 24;

__device__ __forceinline__ uint32_t sub_word(uint32_t w) {
  return uint32_t(g_pool_tables.s[w & 0xFF]) | (uint32_t(g_pool_tables.s[(w >> 8) & 0xFF]) << 8) |
         (uint32_t(g_pool_tables.s[(w >> 16) & 0xFF]) << 16) | (uint32_t(g_pool_tables.s[w >> 24]) << 24);
}

__global__ void expand_keys_kernel(const uint8_t* raw, int nk, uint32_t count, PoolEntry* out) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const uint8_t* key = raw + size_t(k) * 4 * nk;
  const int nr = nk + 6;
  uint32_t w[4 * (kMaxRounds + 1)];
  for (int i = 0; i < nk; ++i)
    w[i] = uint32_t(key[4 * i]) | (uint32_t(key[4 * i + 1]) << 8) | (uint32_t(key[4 * i + 2]) << 16) |
           (uint32_t(key[4 * i + 3]) << 24);
  uint32_t rc = 1;
  for (int i = nk; i < 4 * (nr + 1); ++i) {
    uint32_t t = w[i - 1];
    if (i % nk == 0) {
      t = sub_word((t >> 8) | (t << 24)) ^ rc;  // RotWord moves byte 1 to byte 0
      rc = gf_xtime(uint8_t(rc));
    } else if (nk == 8 && i % 8 == 4) {
      t = sub_word(t);
    }
    w[i] = w[i - nk] ^ t;
  }
  PoolEntry& e = out[k];
  for (int r = 0; r <= kMaxRounds; ++r)
    for (int c = 0; c < 4; ++c) {
      e.enc[r][c] = r <= nr ? w[4 * r + c] : 0u;
      uint32_t d = 0;
      if (r == 0) d = w[4 * nr + c];
      else if (r < nr) d = inv_mix_word(w[4 * (nr - r) + c]);
      else if (r == nr) d = w[c];
      e.dec[r][c] = d;
    }
  e.nr = nr;
  for (int i = 0; i < 7; ++i) e.pad[i] = 0;
}

aes_status check_pool(const aes_keypool* p) {
  if (!p || !p->entries) return set_error(AES_EINVAL, "null or destroyed key pool");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev != p->device) return set_error(AES_EINVAL, "key pool belongs to device %d, current device is %d", p->device, dev);
  return AES_OK;
}

void build_pool_entry_host(const aes_key_schedule& ks, PoolEntry& e) {
  std::memset(&e, 0, sizeof(e));
  const KeyWords enc = enc_key_words(ks, nullptr), dec = dec_key_words(ks, nullptr);
  std::memcpy(e.enc, enc.w, sizeof(e.enc));
  std::memcpy(e.dec, dec.w, sizeof(e.dec));
  e.nr = ks.nr;
}

}  // namespace
}  // namespace aesgb

using namespace aesgb;

extern "C" {

aes_status aes_keypool_create(size_t capacity, aes_keypool** out) {
  clear_error();
  if (!out) return set_error(AES_EINVAL, "null output pointer");
  *out = nullptr;
  if (capacity == 0 || capacity > kMaxPool) return set_error(AES_EINVAL, "capacity must be 1..2^24 (got %zu)", capacity);
  aes_keypool* p = new (std::nothrow) aes_keypool();
  if (!p) return set_error(AES_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { delete p; return cuda_error(e, "cudaGetDevice"); }
  p->nr = new (std::nothrow) int8_t[capacity]();
  p->mu = new (std::nothrow) std::mutex();
  if (!p->nr || !p->mu) {
    delete[] p->nr;
    delete static_cast<std::mutex*>(p->mu);
    delete p;
    return set_error(AES_ENOMEM, "host allocation failed");
  }
  e = cudaMalloc(&p->entries, capacity * sizeof(PoolEntry));
  if (e != cudaSuccess) {
    delete[] p->nr;
    delete static_cast<std::mutex*>(p->mu);
    delete p;
    return set_error(AES_ENOMEM, "key pool cudaMalloc of %zu bytes failed: %s", capacity * sizeof(PoolEntry), cudaGetErrorString(e));
  }
  cudaMemset(p->entries, 0, capacity * sizeof(PoolEntry));
  p->capacity = capacity;
  *out = p;
  return AES_OK;
}

aes_status aes_keypool_load_keys(aes_keypool* pool, uint32_t first, size_t count, const uint8_t* keys,
                                 int key_bits, void* cuda_stream) {
  clear_error();
  aes_status st = check_pool(pool);
  if (st != AES_OK) return st;
  if (key_bits != 128 && key_bits != 192 && key_bits != 256)
    return set_error(AES_EINVAL, "key_bits must be 128, 192 or 256 (got %d)", key_bits);
  if (count == 0) return AES_OK;
  if (!keys) return set_error(AES_EINVAL, "null keys");
  if (size_t(first) >= pool->capacity || count > pool->capacity - first)
    return set_error(AES_EINVAL, "slots %u..%zu exceed the pool capacity %zu", first, size_t(first) + count - 1, pool->capacity);
  const int nk = key_bits / 32;
  const size_t bytes = count * size_t(4 * nk);
  cudaError_t e;
  if (bytes > pool->raw_cap) {
    if (pool->raw) cudaFree(pool->raw);
    pool->raw = nullptr;
    pool->raw_cap = 0;
    if ((e = cudaMalloc(&pool->raw, bytes)) != cudaSuccess)
      return set_error(AES_ENOMEM, "key staging cudaMalloc failed: %s", cudaGetErrorString(e));
    pool->raw_cap = bytes;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if ((e = cudaMemcpyAsync(pool->raw, keys, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync(keys)");
  const unsigned threads = 128, grid = unsigned((count + threads - 1) / threads);
  expand_keys_kernel<<<grid, threads, 0, s>>>(pool->raw, nk, uint32_t(count), pool->entries + first);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "key expansion launch");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "key expansion");
  for (size_t i = 0; i < count; ++i) pool->nr[first + i] = int8_t(nk + 6);
  return AES_OK;
}

aes_status aes_keypool_set(aes_keypool* pool, uint32_t idx, const aes_key_schedule* ks) {
  clear_error();
  aes_status st = check_pool(pool);
  if (st != AES_OK) return st;
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule");
  if (size_t(idx) >= pool->capacity) return set_error(AES_EINVAL, "slot %u out of range (capacity %zu)", idx, pool->capacity);
  PoolEntry e;
  build_pool_entry_host(*ks, e);
  cudaError_t ce = cudaMemcpy(pool->entries + idx, &e, sizeof(e), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return cuda_error(ce, "cudaMemcpy(pool entry)");
  pool->nr[idx] = int8_t(ks->nr);
  return AES_OK;
}

int aes_keypool_rounds(const aes_keypool* pool, uint32_t idx) {
  if (!pool || !pool->nr || size_t(idx) >= pool->capacity) return 0;
  return pool->nr[idx];
}

aes_status aes_batch_destroy(aes_batch* b);

aes_status aes_keypool_destroy(aes_keypool* pool) {
  clear_error();
  if (!pool) return AES_OK;
  if (pool->internal) aes_batch_destroy(pool->internal);
  aesgb::cbc_batched_release(pool);
  if (pool->entries) cudaFree(pool->entries);
  if (pool->raw) cudaFree(pool->raw);
  delete[] pool->nr;
  delete static_cast<std::mutex*>(pool->mu);
  delete pool;
  return AES_OK;
}

}  // extern "C"
