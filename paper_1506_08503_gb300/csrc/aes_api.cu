// aes_api.cu -- the C ABI entry points for keys and plain block encryption/decryption,
// plus the library's error and device bookkeeping.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "aes_internal.cuh"

namespace aesgb {

// ---- errors -------------------------------------------------------------------------
namespace {
thread_local char t_err[512] = {0};
}

aes_status set_error(aes_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  return st;
}

aes_status cuda_error(cudaError_t e, const char* what) {
  return set_error(AES_ECUDA, "%s: %s (%d)", what, cudaGetErrorString(e), int(e));
}

void clear_error() { t_err[0] = 0; }

// ---- device facts ---------------------------------------------------------------------
namespace {
constexpr int kMaxDevices = 64;
DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;
}  // namespace

const DeviceInfo* current_device_info() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { cuda_error(e, "cudaGetDevice"); return nullptr; }
  if (dev < 0 || dev >= kMaxDevices) { set_error(AES_ECUDA, "device ordinal %d out of range", dev); return nullptr; }
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo& d = g_dev[dev];
  if (d.device == dev) return &d;
  int sms = 0, optin = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) {
    cuda_error(e, "cudaDeviceGetAttribute");
    return nullptr;
  }
  cudaDeviceProp p;
  if ((e = cudaGetDeviceProperties(&p, dev)) != cudaSuccess) { cuda_error(e, "cudaGetDeviceProperties"); return nullptr; }
  int pageable = 0, host_tables = 0;
  if ((e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev)) != cudaSuccess) {
    cuda_error(e, "cudaDeviceGetAttribute");
    return nullptr;
  }
  d.sms = sms;
  d.smem_optin = optin;
  d.host_direct = pageable == 1 && host_tables == 1;
  std::snprintf(d.name, sizeof(d.name), "%s", p.name);
  d.device = dev;
  return &d;
}

namespace {
struct KernelFact {
  int device;
  const void* fn;
  size_t smem;
  int threads;  // 0 for the shared-memory attribute, else an occupancy entry
  int value;
};
std::mutex g_fact_mu;
std::vector<KernelFact> g_facts;
}  // namespace

aes_status ensure_kernel_smem(const void* fn, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_fact_mu);
  for (const KernelFact& f : g_facts)
    if (f.device == dev && f.fn == fn && f.threads == 0 && f.smem >= bytes) return AES_OK;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes))) != cudaSuccess)
    return cuda_error(e, "cudaFuncSetAttribute");
  g_facts.push_back(KernelFact{dev, fn, bytes, 0, 0});
  return AES_OK;
}

aes_status kernel_ctas_per_sm(const void* fn, int threads, size_t smem, int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_fact_mu);
  for (const KernelFact& f : g_facts)
    if (f.device == dev && f.fn == fn && f.threads == threads && f.smem == smem) {
      *out = f.value;
      return AES_OK;
    }
  int n = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem)) != cudaSuccess)
    return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  g_facts.push_back(KernelFact{dev, fn, smem, threads, n});
  *out = n;
  return AES_OK;
}

// ---- keys -------------------------------------------------------------------------------
namespace {

constexpr FieldTables kHostTables = make_field_tables();

uint32_t load_word(const uint8_t* p) {
  return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) | (uint32_t(p[3]) << 24);
}

}  // namespace

bool schedule_ok(const aes_key_schedule* ks) {
  return ks && (ks->nr == 10 || ks->nr == 12 || ks->nr == 14);
}

KeyWords enc_key_words(const aes_key_schedule& ks, const uint8_t* iv) {
  KeyWords kw{};
  for (int r = 0; r <= ks.nr; ++r)
    for (int c = 0; c < 4; ++c) kw.w[r][c] = load_word(ks.rk[r] + 4 * c);
  if (iv)
    for (int c = 0; c < 4; ++c) kw.w[0][c] ^= load_word(iv + 4 * c);
  return kw;
}

KeyWords dec_key_words(const aes_key_schedule& ks, const uint8_t* iv) {
  KeyWords kw{};
  const int nr = ks.nr;
  for (int c = 0; c < 4; ++c) kw.w[0][c] = load_word(ks.rk[nr] + 4 * c);
  for (int r = 1; r < nr; ++r)
    for (int c = 0; c < 4; ++c) kw.w[r][c] = inv_mix_word(load_word(ks.rk[nr - r] + 4 * c));
  for (int c = 0; c < 4; ++c) kw.w[nr][c] = load_word(ks.rk[0] + 4 * c) ^ (iv ? load_word(iv + 4 * c) : 0u);
  return kw;
}

}  // namespace aesgb

using namespace aesgb;

extern "C" {

const char* aes_last_error(void) { return t_err; }

const char* aes_version(void) { return "aesgb 1.0 sm_103a"; }

// Key expansion in words w[0..4(nr+1)): w[i] = w[i-nk] ^ t with t built from w[i-1] by
// RotWord+SubWord+Rcon every nk words (App. A3 for nk = 4) and SubWord alone at i = 4 mod 8
// when nk = 8 (FIPS-197 Section 5.2).
aes_status aes_key_expand(const uint8_t* key, int key_bits, aes_key_schedule* out) {
  clear_error();
  if (!key || !out) return set_error(AES_EINVAL, "aes_key_expand: null pointer");
  int nk;
  switch (key_bits) {
    case 128: nk = 4; break;
    case 192: nk = 6; break;
    case 256: nk = 8; break;
    default: return set_error(AES_EINVAL, "aes_key_expand: key_bits must be 128, 192 or 256 (got %d)", key_bits);
  }
  const int nr = nk + 6;
  uint8_t w[4 * (kMaxRounds + 1)][4];
  std::memcpy(w, key, size_t(4 * nk));
  uint8_t rc = 1;  // x^(i/nk - 1), advanced by xtime
  for (int i = nk; i < 4 * (nr + 1); ++i) {
    uint8_t t[4] = {w[i - 1][0], w[i - 1][1], w[i - 1][2], w[i - 1][3]};
    if (i % nk == 0) {
      const uint8_t t0 = t[0];
      t[0] = uint8_t(kHostTables.s[t[1]] ^ rc);
      t[1] = kHostTables.s[t[2]];
      t[2] = kHostTables.s[t[3]];
      t[3] = kHostTables.s[t0];
      rc = gf_xtime(rc);
    } else if (nk == 8 && i % 8 == 4) {
      for (int j = 0; j < 4; ++j) t[j] = kHostTables.s[t[j]];
    }
    for (int j = 0; j < 4; ++j) w[i][j] = uint8_t(w[i - nk][j] ^ t[j]);
  }
  std::memset(out, 0, sizeof(*out));
  out->nr = nr;
  std::memcpy(out->rk, w, size_t(16 * (nr + 1)));
  return AES_OK;
}

aes_status aes_crypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                            void* d_out, size_t nblocks, int dir, int impl, void* cuda_stream) {
  clear_error();
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (impl != AES_IMPL_AUTO && impl != AES_IMPL_TTABLE && impl != AES_IMPL_BITSLICE)
    return set_error(AES_EINVAL, "unknown impl %d", impl);
  if (nblocks == 0) return AES_OK;
  if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  if (nblocks > (SIZE_MAX >> 5)) return set_error(AES_EINVAL, "nblocks too large");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  const uintptr_t bytes = uintptr_t(nblocks) * 16u;
  if (a != b && a < b + bytes && b < a + bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TTConfig cfg;
  if (impl == AES_IMPL_AUTO) {
    bool pinned = false;
    if (!tuned_choice(dir, ks->nr, &impl, &cfg, &pinned)) impl = AES_IMPL_TTABLE;
    if (!pinned && nblocks <= kSmallCallBlocks) {
      // a small call: the tables come from global memory, no shared-memory fill per CTA
      const KeyWords kw = dir == AES_ENCRYPT ? enc_key_words(*ks, iv) : dec_key_words(*ks, iv);
      return launch_small(dir, ks->nr, kw, d_in, d_out, nblocks, st);
    }
  }
  if (impl == AES_IMPL_BITSLICE) return launch_bitslice(dir, *ks, iv, d_in, d_out, nblocks, st, BSConfig{});
  const KeyWords kw = dir == AES_ENCRYPT ? enc_key_words(*ks, iv) : dec_key_words(*ks, iv);
  return launch_ttable(dir, ks->nr, kw, d_in, d_out, nblocks, st, cfg);
}

aes_status aes_encrypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                              void* d_out, size_t nblocks, void* cuda_stream) {
  return aes_crypt_blocks(ks, iv, d_in, d_out, nblocks, AES_ENCRYPT, AES_IMPL_AUTO, cuda_stream);
}

aes_status aes_decrypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                              void* d_out, size_t nblocks, void* cuda_stream) {
  return aes_crypt_blocks(ks, iv, d_in, d_out, nblocks, AES_DECRYPT, AES_IMPL_AUTO, cuda_stream);
}

}  // extern "C"
