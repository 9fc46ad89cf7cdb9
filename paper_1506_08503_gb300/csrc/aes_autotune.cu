// aes_autotune.cu -- the launch tuner of the single-key path: which kernel family (T-tables
// or the bitsliced circuit, whose width is 32 blocks per thread) and, for the T-tables, which
// CTA size and blocks in flight per thread aes_crypt_blocks uses when asked for
// AES_IMPL_AUTO.  The tuner times every compiled candidate on the caller's buffers and keeps
// the fastest per (device, direction, round count) for the rest of the process; a JSON file
// can carry the result across processes, keyed by device name and a size signature.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "aes_internal.cuh"
#include "aesgb_testing.h"

namespace aesgb {
namespace {

struct Candidate {
  int impl, threads, unroll;
};
// every compiled T-table shape (see tt::select_config) and the bitsliced kernel
constexpr Candidate kCandidates[] = {{AES_IMPL_TTABLE, 512, 2},  {AES_IMPL_TTABLE, 512, 1},  {AES_IMPL_TTABLE, 512, 4},
                                     {AES_IMPL_TTABLE, 256, 4},  {AES_IMPL_TTABLE, 1024, 1}, {AES_IMPL_TTABLE, 1024, 2},
                                     {AES_IMPL_TTABLE, 768, 2},
                                     {AES_IMPL_BITSLICE, 128, 32}};
constexpr int kDevices = 64;

struct Tuned {
  bool set = false;
  bool pinned = false;  // set by aes_set_auto_choice: serves every size, small calls too
  Candidate c{};
};
std::mutex g_mu;
Tuned g_tuned[kDevices][2][3];  // device, direction, (nr - 10) / 2

bool valid(const Candidate& c) {
  for (const Candidate& k : kCandidates)
    if (k.impl == c.impl && k.threads == c.threads && k.unroll == c.unroll) return true;
  return false;
}

aes_status run(const Candidate& c, const aes_key_schedule& ks, const void* in, void* out, size_t n, int dir,
               cudaStream_t st) {
  if (c.impl == AES_IMPL_BITSLICE) return launch_bitslice(dir, ks, nullptr, in, out, n, st, BSConfig{});
  TTConfig cfg;
  cfg.threads = c.threads;
  cfg.unroll = c.unroll;
  const KeyWords kw = dir == AES_ENCRYPT ? enc_key_words(ks, nullptr) : dec_key_words(ks, nullptr);
  return launch_ttable(dir, ks.nr, kw, in, out, n, st, cfg);
}

std::string read_file(const char* path) {
  std::string out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, k);
  std::fclose(f);
  return out;
}

// The cache is one flat JSON object: {"signature": {"impl": I, "threads": T, "unroll": U, "us": x}, ...}
bool cache_lookup(const std::string& text, const std::string& sig, Candidate* c) {
  const size_t p = text.find("\"" + sig + "\"");
  if (p == std::string::npos) return false;
  const size_t e = text.find('}', p);
  int v[3];
  const char* keys[3] = {"\"impl\":", "\"threads\":", "\"unroll\":"};
  for (int i = 0; i < 3; ++i) {
    const size_t q = text.find(keys[i], p);
    if (q == std::string::npos || q > e || std::sscanf(text.c_str() + q + std::strlen(keys[i]), "%d", &v[i]) != 1) return false;
  }
  *c = Candidate{v[0], v[1], v[2]};
  return valid(*c);
}

void cache_store(const char* path, const std::string& text, const std::string& sig, const Candidate& c, double us) {
  char entry[512];
  std::snprintf(entry, sizeof(entry), "\"%s\": {\"impl\": %d, \"threads\": %d, \"unroll\": %d, \"us\": %.1f}", sig.c_str(),
                c.impl, c.threads, c.unroll, us);
  std::string body = text;
  const size_t close = body.rfind('}');
  if (body.find('{') == std::string::npos || close == std::string::npos) {
    body = std::string("{\n  ") + entry + "\n}\n";
  } else {
    const bool empty = body.find('"') == std::string::npos;
    body = body.substr(0, close);
    while (!body.empty() && (body.back() == '\n' || body.back() == ' ')) body.pop_back();
    body += (empty ? "\n  " : ",\n  ") + std::string(entry) + "\n}\n";
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  std::fwrite(body.data(), 1, body.size(), f);
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

}  // namespace

bool tuned_choice(int dir, int nr, int* impl, TTConfig* cfg, bool* pinned) {
  int dev = 0;
  if (pinned) *pinned = false;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  const Tuned& t = g_tuned[dev][dir == AES_DECRYPT][(nr - 10) / 2];
  if (!t.set) return false;
  *impl = t.c.impl;
  cfg->threads = t.c.threads;
  cfg->unroll = t.c.unroll;
  if (pinned) *pinned = t.pinned;
  return true;
}

}  // namespace aesgb

using namespace aesgb;

extern "C" aes_status aes_autotune_blocks(const aes_key_schedule* ks, const void* d_in, void* d_out, size_t nblocks,
                                          int dir, const char* cache_path, int* impl, int* threads, int* unroll,
                                          void* cuda_stream) {
  clear_error();
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (nblocks == 0) return set_error(AES_EINVAL, "nothing to time (nblocks = 0)");
  if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  if (nblocks > (SIZE_MAX >> 5)) return set_error(AES_EINVAL, "nblocks too large");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  const uintptr_t bytes = uintptr_t(nblocks) * 16u;
  if (a != b && a < b + bytes && b < a + bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kDevices) return set_error(AES_ECUDA, "device ordinal %d out of range", dev);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  char sigbuf[400];
  std::snprintf(sigbuf, sizeof(sigbuf), "%s|%s|nr%d|log2n%d", di->name, dir == AES_ENCRYPT ? "enc" : "dec", ks->nr,
                int(std::floor(std::log2(double(nblocks)))));
  const std::string sig = sigbuf;
  std::string text = cache_path ? read_file(cache_path) : std::string();
  Candidate best{};
  double best_us = -1.0;
  if (!(cache_path && cache_lookup(text, sig, &best))) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return cuda_error(e, "cudaEventCreate");
    }
    aes_status rc = AES_OK;
    for (const Candidate& c : kCandidates) {
      if ((rc = run(c, *ks, d_in, d_out, nblocks, dir, st)) != AES_OK) break;  // warm-up
      constexpr int kReps = 3;
      cudaEventRecord(e0, st);
      for (int r = 0; r < kReps && rc == AES_OK; ++r) rc = run(c, *ks, d_in, d_out, nblocks, dir, st);
      cudaEventRecord(e1, st);
      if (rc != AES_OK) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_error(e, "cudaEventSynchronize"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1e3 * ms / kReps;
      if (best_us < 0 || us < best_us) {
        best_us = us;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AES_OK) return rc;
    if (cache_path) cache_store(cache_path, text, sig, best, best_us);
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    Tuned& t = g_tuned[dev][dir == AES_DECRYPT][(ks->nr - 10) / 2];
    t.set = true;
    t.pinned = false;
    t.c = best;
  }
  if (impl) *impl = best.impl;
  if (threads) *threads = best.threads;
  if (unroll) *unroll = best.unroll;
  return AES_OK;
}

extern "C" aes_status aes_set_auto_choice(int dir, int nr, int impl, int threads, int unroll) {
  clear_error();
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (nr != 10 && nr != 12 && nr != 14) return set_error(AES_EINVAL, "nr must be 10, 12 or 14");
  const Candidate c{impl, threads, unroll};
  if (impl != AES_IMPL_AUTO && !valid(c))
    return set_error(AES_EINVAL, "(impl %d, %d threads, %d per thread) is not a compiled candidate", impl, threads, unroll);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kDevices) return set_error(AES_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  Tuned& t = g_tuned[dev][dir == AES_DECRYPT][(nr - 10) / 2];
  if (impl == AES_IMPL_AUTO) {  // back to the default: no tuned or pinned choice
    t = Tuned{};
    return AES_OK;
  }
  t.set = true;
  t.pinned = true;
  t.c = c;
  return AES_OK;
}

extern "C" int aes_testing_tune_cache_store(const char* path, const char* sig, int impl, int threads, int unroll,
                                            double us) {
  if (!path || !sig) return -1;
  cache_store(path, read_file(path), sig, Candidate{impl, threads, unroll}, us);
  return 0;
}

extern "C" int aes_testing_tune_cache_lookup(const char* path, const char* sig, int* impl, int* threads, int* unroll) {
  if (!path || !sig || !impl || !threads || !unroll) return -1;
  Candidate c{};
  if (!cache_lookup(read_file(path), sig, &c)) return 0;
  *impl = c.impl;
  *threads = c.threads;
  *unroll = c.unroll;
  return 1;
}
