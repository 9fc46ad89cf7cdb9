// aes_batched.cu -- host side of the batched launch: descriptor staging, the cached CUDA
// graph that replays the two-direction kernel, the autotuner and aes_crypt_batched.
//
// Per run the host splits the messages by direction, drops empty ones, writes 32-byte
// descriptors plus each message's first block in the direction's concatenated block space
// into pinned staging, cuts each direction into per-warp slices of equal work (blocks x
// rounds), splits the CTAs between the directions in proportion to their work, copies all of
// it to the device on the batch's own copy stream (so the upload overlaps whatever the
// caller's stream is still running, e.g. the previous batch), and launches the graph [one
// kernel, both directions] on the caller's stream behind that copy.  The graph is built once
// per shape; later runs patch the kernel arguments (cudaGraphExecKernelNodeSetParams) when
// they change.  Two staging/device buffer pairs alternate; a run waits for the run that used
// its pair two calls ago, so descriptors are never overwritten while a kernel reads them.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "aes_internal.cuh"
#include "aesgb_testing.h"

namespace {

using namespace aesgb;

constexpr size_t kMaxMsgs = size_t(1) << 24;

struct Shape {
  int threads, bpl;
};
// (CTA threads, blocks each lane enciphers per window)
// (768, 1) is compiled for AES-128 work only; a launch with other round counts at that shape
// takes (512, 1).
constexpr Shape kShapes[] = {{512, 1}, {512, 2}, {512, 4}, {384, 4}, {256, 4}, {768, 1}};
constexpr int kMaxShapeThreads = 768;

struct Slot {
  uint8_t* host = nullptr;  // pinned staging
  uint8_t* dev = nullptr;
  cudaEvent_t done = nullptr;    // the kernels that read this slot have finished
  cudaEvent_t copied = nullptr;  // this slot's descriptors are on the device
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel = nullptr;
};

struct Layout {
  size_t enc_msgs, dec_msgs, enc_start, dec_start, enc_gb, dec_gb, enc_warp, dec_warp, end, enc_iv, dec_iv, end_iv;
};

// wmax: most warps a launch can have (SMs x the largest shape's threads / 32)
Layout layout(size_t nenc, size_t ndec, size_t wmax) {
  Layout l;
  l.enc_msgs = 0;
  l.dec_msgs = l.enc_msgs + nenc * sizeof(BatchMsg);
  l.enc_start = l.dec_msgs + ndec * sizeof(BatchMsg);
  l.dec_start = l.enc_start + (nenc + 1) * sizeof(uint64_t);
  l.enc_gb = l.dec_start + (ndec + 1) * sizeof(uint64_t);
  l.dec_gb = l.enc_gb + (wmax + 1) * sizeof(uint64_t);
  l.enc_warp = l.dec_gb + (wmax + 1) * sizeof(uint64_t);
  l.dec_warp = l.enc_warp + wmax * sizeof(uint32_t);
  l.end = l.dec_warp + wmax * sizeof(uint32_t);
  // per-message IVs (uploaded only by runs that carry them), 16-byte aligned
  l.enc_iv = (l.end + 15) & ~size_t(15);
  l.dec_iv = l.enc_iv + nenc * 16;
  l.end_iv = l.dec_iv + ndec * 16;
  return l;
}

}  // namespace

namespace aesgb {

// Work of a direction in round-blocks (a block of an Nr-round key costs Nr).
uint64_t work_of(const BatchMsg* m, size_t n, const int8_t* rounds) {
  uint64_t w = 0;
  for (size_t i = 0; i < n; ++i) w += m[i].nblocks * uint64_t(rounds[m[i].key_idx]);
  return w;
}

// Cuts a direction's block space into nw slices of equal work: warp w starts at the block
// where the running work reaches floor(W * w / nw).  gb[w] is that block (gb[nw] = the
// direction's total), msg[w] the message holding it.  Targets advance incrementally.
void weighted_slices(const BatchMsg* m, const uint64_t* start, size_t n, const int8_t* rounds, uint64_t W,
                     uint64_t nw, uint64_t* gb, uint32_t* msg) {
  if (nw == 0) return;
  const uint64_t step = W / nw, rem = W % nw;
  uint64_t t = 0, r = 0, acc = 0;  // acc: work before message i
  size_t i = 0;
  for (uint64_t w = 0; w < nw; ++w) {
    uint64_t rw = uint64_t(rounds[m[i].key_idx]);
    while (i + 1 < n && acc + m[i].nblocks * rw <= t) {
      acc += m[i].nblocks * rw;
      ++i;
      rw = uint64_t(rounds[m[i].key_idx]);
    }
    const uint64_t off = std::min<uint64_t>((t - acc) / rw, m[i].nblocks - 1);
    gb[w] = start[i] + off;
    msg[w] = uint32_t(i);
    t += step;
    r += rem;
    if (r >= nw) {
      ++t;
      r -= nw;
    }
  }
  gb[nw] = start[n];
}

}  // namespace aesgb

struct aes_batch {
  aes_keypool* pool = nullptr;
  int device = -1;
  size_t max_msgs = 0;
  size_t bytes = 0;
  size_t wmax = 0;
  // default shape (the autotuner may change it): 768 threads, 1 block per lane where a launch's
  // work is all AES-128 (0.84-0.85 of the plain kernel on the 4096-message workload, against
  // 0.80-0.82 for 512 x 1), else 512 x 1 (on the served mix: 1 ~ 2 > 4 blocks per lane)
  int threads = 768, bpl = 1;
  Slot slot[2];
  int next = 0;
  cudaStream_t copy_stream = nullptr;
  std::mutex mu;
};

namespace {

void free_slot(Slot& s) {
  if (s.exec) cudaGraphExecDestroy(s.exec);
  if (s.graph) cudaGraphDestroy(s.graph);
  if (s.done) cudaEventDestroy(s.done);
  if (s.copied) cudaEventDestroy(s.copied);
  if (s.dev) cudaFree(s.dev);
  if (s.host) cudaFreeHost(s.host);
  s = Slot{};
}

struct KernelArgs {
  uint64_t in;
  uint64_t out;
  BatchDir be, bd;
  const PoolEntry* pool;
  uint32_t ge;
  void* ptrs[6];
  void fix() {
    ptrs[0] = &in;
    ptrs[1] = &out;
    ptrs[2] = &be;
    ptrs[3] = &bd;
    ptrs[4] = &pool;
    ptrs[5] = &ge;
  }
};

cudaKernelNodeParams kernel_params(TTDualFn fn, unsigned grid, int threads, size_t smem, KernelArgs& a) {
  a.fix();
  cudaKernelNodeParams p{};
  p.func = reinterpret_cast<void*>(fn);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(unsigned(threads));
  p.sharedMemBytes = unsigned(smem);
  p.kernelParams = a.ptrs;
  p.extra = nullptr;
  return p;
}

aes_status build_graph(Slot& s, const cudaKernelNodeParams& p) {
  if (s.exec) { cudaGraphExecDestroy(s.exec); s.exec = nullptr; }
  if (s.graph) { cudaGraphDestroy(s.graph); s.graph = nullptr; }
  cudaError_t e;
  if ((e = cudaGraphCreate(&s.graph, 0)) != cudaSuccess) return cuda_error(e, "cudaGraphCreate");
  if ((e = cudaGraphAddKernelNode(&s.kernel, s.graph, nullptr, 0, &p)) != cudaSuccess) return cuda_error(e, "cudaGraphAddKernelNode");
  if ((e = cudaGraphInstantiate(&s.exec, s.graph, 0)) != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
  return AES_OK;
}

// The kernels' dynamic shared-memory limit, raised once per device and kernel.
aes_status ensure_smem_attr(TTDualFn f, size_t smem) { return ensure_kernel_smem(reinterpret_cast<const void*>(f), smem); }

}  // namespace

namespace aesgb {

// Writes nenc + ndec descriptors through `fill` into the next staging slot, computes the
// per-direction block starts and launches the graph on `stream`.  Caller holds b->mu.
aes_status batch_launch_descs(aes_batch* b, size_t nenc, size_t ndec, const DescFill& fill, bool with_ivs,
                              uint64_t in_base, uint64_t out_base, cudaStream_t stream) {
  cudaError_t e;
  if (nenc + ndec > b->max_msgs) return set_error(AES_EINVAL, "%zu messages exceed the batch capacity %zu", nenc + ndec, b->max_msgs);
  Slot& s = b->slot[b->next];
  b->next ^= 1;
  if ((e = cudaEventSynchronize(s.done)) != cudaSuccess) return cuda_error(e, "waiting for a previous batch");
  const Layout L = layout(nenc, ndec, b->wmax);
  uint8_t* h = s.host;
  BatchMsg* em = reinterpret_cast<BatchMsg*>(h + L.enc_msgs);
  BatchMsg* dm = reinterpret_cast<BatchMsg*>(h + L.dec_msgs);
  uint64_t* es = reinterpret_cast<uint64_t*>(h + L.enc_start);
  uint64_t* ds = reinterpret_cast<uint64_t*>(h + L.dec_start);
  uint4* eiv = with_ivs ? reinterpret_cast<uint4*>(h + L.enc_iv) : nullptr;
  uint4* div = with_ivs ? reinterpret_cast<uint4*>(h + L.dec_iv) : nullptr;
  fill(em, dm, eiv, div);
  uint64_t te = 0, td = 0;
  for (size_t i = 0; i < nenc; ++i) { es[i] = te; te += em[i].nblocks; }
  for (size_t i = 0; i < ndec; ++i) { ds[i] = td; td += dm[i].nblocks; }
  es[nenc] = te;
  ds[ndec] = td;

  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  const int8_t* rounds = b->pool->nr;
  const uint64_t we = work_of(em, nenc, rounds), wd = work_of(dm, ndec, rounds);
  // AES-128 throughout a direction (work = 10 x blocks, as no key has fewer rounds) takes the
  // specialised kernel; an empty direction takes the other's count
  int nre = te && we == 10 * te ? 10 : 0, nrd = td && wd == 10 * td ? 10 : 0;
  if (!te) nre = nrd;
  if (!td) nrd = nre;
  int threads = b->threads, bpl = b->bpl;
  TTDualFn fn = ttable_batched_dual(threads, bpl, nre, nrd);
  if (!fn && threads == 768) {
    threads = 512;
    bpl = 1;
    fn = ttable_batched_dual(threads, bpl, nre, nrd);
  }
  if (!fn) return set_error(AES_EINVAL, "shape (%d threads, %d blocks per lane) is not compiled", threads, bpl);
  const size_t smem = ttable_smem_bytes(AES_DECRYPT);
  aes_status ast = ensure_smem_attr(fn, smem);
  if (ast != AES_OK) return ast;
  // one CTA per SM (fewer when there is less than one block per thread), split between the
  // directions in proportion to their work in round-blocks
  const uint64_t per_cta = uint64_t(threads);
  uint64_t G = std::max<uint64_t>(1, std::min<uint64_t>(di->sms, (te + td + per_cta - 1) / per_cta));
  if (te && td) G = std::max<uint64_t>(G, 2);
  uint64_t ge = 0;
  if (!td) ge = G;
  else if (te) ge = std::min<uint64_t>(G - 1, std::max<uint64_t>(1, (G * we + (we + wd) / 2) / (we + wd)));
  const uint64_t gd = G - ge;
  const uint64_t wpc = uint64_t(threads / 32), nwe = ge * wpc, nwd = gd * wpc;
  if (nwe > b->wmax || nwd > b->wmax) return set_error(AES_ECUDA, "device has more SMs than the batch was sized for");
  weighted_slices(em, es, nenc, rounds, we, te ? nwe : 0, reinterpret_cast<uint64_t*>(h + L.enc_gb),
                  reinterpret_cast<uint32_t*>(h + L.enc_warp));
  weighted_slices(dm, ds, ndec, rounds, wd, td ? nwd : 0, reinterpret_cast<uint64_t*>(h + L.dec_gb),
                  reinterpret_cast<uint32_t*>(h + L.dec_warp));
  KernelArgs a{in_base, out_base,
               BatchDir{reinterpret_cast<const BatchMsg*>(s.dev + L.enc_msgs), reinterpret_cast<const uint64_t*>(s.dev + L.enc_start),
                        reinterpret_cast<const uint32_t*>(s.dev + L.enc_warp), te, uint32_t(nenc), 0u,
                        reinterpret_cast<const uint64_t*>(s.dev + L.enc_gb),
                        with_ivs ? reinterpret_cast<const uint4*>(s.dev + L.enc_iv) : nullptr},
               BatchDir{reinterpret_cast<const BatchMsg*>(s.dev + L.dec_msgs), reinterpret_cast<const uint64_t*>(s.dev + L.dec_start),
                        reinterpret_cast<const uint32_t*>(s.dev + L.dec_warp), td, uint32_t(ndec), 0u,
                        reinterpret_cast<const uint64_t*>(s.dev + L.dec_gb),
                        with_ivs ? reinterpret_cast<const uint4*>(s.dev + L.dec_iv) : nullptr},
               b->pool->entries, uint32_t(ge), {}};
  const cudaKernelNodeParams p = kernel_params(fn, unsigned(G), threads, smem, a);
  if (!s.exec) {  // a later launch with another kernel or shape updates the node in place
    aes_status st = build_graph(s, p);
    if (st != AES_OK) return st;
  } else if ((e = cudaGraphExecKernelNodeSetParams(s.exec, s.kernel, &p)) != cudaSuccess) {
    return cuda_error(e, "cudaGraphExecKernelNodeSetParams");
  }
  if ((e = cudaMemcpyAsync(s.dev, s.host, with_ivs ? L.end_iv : L.end, cudaMemcpyHostToDevice, b->copy_stream)) !=
      cudaSuccess)
    return cuda_error(e, "descriptor upload");
  if ((e = cudaEventRecord(s.copied, b->copy_stream)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(stream, s.copied, 0)) != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
  if ((e = cudaGraphLaunch(s.exec, stream)) != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  if ((e = cudaEventRecord(s.done, stream)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  return AES_OK;
}

}  // namespace aesgb

namespace {

aes_status run_locked(aes_batch* b, const aes_msg* msgs, size_t nmsgs, const void* d_in, void* d_out,
                      size_t buf_bytes, cudaStream_t stream, const uint8_t* ivs = nullptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev != b->device) return set_error(AES_EINVAL, "batch belongs to device %d, current device is %d", b->device, dev);
  if (nmsgs > b->max_msgs) return set_error(AES_EINVAL, "%zu messages exceed the batch capacity %zu", nmsgs, b->max_msgs);
  if (nmsgs && !msgs) return set_error(AES_EINVAL, "null message array");
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
    return set_error(AES_EINVAL, "buffers must be 16-byte aligned");
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), o = reinterpret_cast<uintptr_t>(d_out);
  if (a != o && a < o + buf_bytes && o < a + buf_bytes)
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  const aes_keypool* pool = b->pool;
  size_t nenc = 0, ndec = 0;
  for (size_t i = 0; i < nmsgs; ++i) {
    const aes_msg& m = msgs[i];
    if (m.dir != AES_ENCRYPT && m.dir != AES_DECRYPT) return set_error(AES_EINVAL, "message %zu: bad dir %u", i, m.dir);
    if ((m.offset | m.length) & 15u) return set_error(AES_EINVAL, "message %zu: offset and length must be multiples of 16", i);
    if (m.offset > buf_bytes || m.length > buf_bytes - m.offset)
      return set_error(AES_EINVAL, "message %zu: [%llu, +%llu) leaves the %zu-byte buffers", i,
                       (unsigned long long)m.offset, (unsigned long long)m.length, buf_bytes);
    if (m.length == 0) continue;
    if (!d_in || !d_out) return set_error(AES_EINVAL, "null buffer");
    if (size_t(m.key_idx) >= pool->capacity || pool->nr[m.key_idx] == 0)
      return set_error(AES_EINVAL, "message %zu: key slot %u is not loaded", i, m.key_idx);
    (m.dir == AES_ENCRYPT ? nenc : ndec)++;
  }
  auto fill = [&](BatchMsg* em, BatchMsg* dm, uint4* eiv, uint4* div) {
    size_t ie = 0, id = 0;
    for (size_t i = 0; i < nmsgs; ++i) {
      const aes_msg& m = msgs[i];
      if (m.length == 0) continue;
      const BatchMsg d{m.key_idx, 0u, m.offset / 16, m.offset / 16, m.length / 16};
      if (m.dir == AES_ENCRYPT) {
        if (eiv) std::memcpy(eiv + ie, ivs + 16 * i, 16);
        em[ie++] = d;
      } else {
        if (div) std::memcpy(div + id, ivs + 16 * i, 16);
        dm[id++] = d;
      }
    }
  };
  return batch_launch_descs(b, nenc, ndec, fill, ivs != nullptr, reinterpret_cast<uint64_t>(d_in),
                            reinterpret_cast<uint64_t>(d_out), stream);
}

// The round count every message of each direction has, as batch_launch_descs derives it from
// the descriptors (10 for AES-128 throughout, else 0; an empty direction takes the other's).
void round_classes(const aes_keypool* pool, const aes_msg* msgs, size_t n, int* nre, int* nrd) {
  bool e_any = false, d_any = false, e10 = true, d10 = true;
  for (size_t i = 0; i < n; ++i) {
    if (msgs[i].length == 0) continue;
    const bool ten = size_t(msgs[i].key_idx) < pool->capacity && pool->nr[msgs[i].key_idx] == 10;
    if (msgs[i].dir == AES_ENCRYPT) {
      e_any = true;
      e10 &= ten;
    } else {
      d_any = true;
      d10 &= ten;
    }
  }
  *nre = e_any && e10 ? 10 : 0;
  *nrd = d_any && d10 ? 10 : 0;
  if (!e_any) *nre = *nrd;
  if (!d_any) *nrd = *nre;
}

bool shape_compiled(int threads, int bpl) {
  for (const Shape& sh : kShapes)
    if (sh.threads == threads && sh.bpl == bpl) return true;
  return false;
}

// ---- autotune cache: a flat JSON object {"signature": {"threads": T, "blocks_per_lane": U, "us": x}, ...}
std::string read_file(const char* path) {
  std::string out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, n);
  std::fclose(f);
  return out;
}

bool cache_lookup(const std::string& text, const std::string& sig, int* threads, int* bpl) {
  const std::string key = "\"" + sig + "\"";
  size_t p = text.find(key);
  if (p == std::string::npos) return false;
  int t = 0, u = 0;
  const size_t pt = text.find("\"threads\":", p), pu = text.find("\"blocks_per_lane\":", p);
  if (pt == std::string::npos || pu == std::string::npos) return false;
  if (std::sscanf(text.c_str() + pt + 10, "%d", &t) != 1 || std::sscanf(text.c_str() + pu + 18, "%d", &u) != 1) return false;
  if (!shape_compiled(t, u)) return false;
  *threads = t;
  *bpl = u;
  return true;
}

void cache_store(const char* path, const std::string& text, const std::string& sig, int threads, int bpl, double us) {
  char entry[512];
  std::snprintf(entry, sizeof(entry), "\"%s\": {\"threads\": %d, \"blocks_per_lane\": %d, \"us\": %.1f}", sig.c_str(), threads, bpl, us);
  std::string body = text;
  const size_t close = body.rfind('}');
  if (body.empty() || close == std::string::npos || body.find('{') == std::string::npos) body = std::string("{\n  ") + entry + "\n}\n";
  else {
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

std::string signature(const DeviceInfo* di, const aes_msg* msgs, size_t n) {
  uint64_t blocks = 0, enc = 0;
  for (size_t i = 0; i < n; ++i) {
    blocks += msgs[i].length / 16;
    if (msgs[i].dir == AES_ENCRYPT) enc += msgs[i].length / 16;
  }
  // bucket sizes to powers of two so that nearby workloads share an entry
  auto lg = [](uint64_t v) { int b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
  char buf[400];
  std::snprintf(buf, sizeof(buf), "%s|msgs=2^%d|blocks=2^%d|enc=%d%%", di->name, lg(n), lg(blocks),
                blocks ? int(100 * enc / blocks) : 0);
  return buf;
}

}  // namespace

using namespace aesgb;

extern "C" {

aes_status aes_batch_destroy(aes_batch* b) {
  clear_error();
  if (!b) return AES_OK;
  for (Slot& s : b->slot) {
    if (s.done) cudaEventSynchronize(s.done);
    free_slot(s);
  }
  if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
  delete b;
  return AES_OK;
}

aes_status aes_batch_create(aes_keypool* pool, size_t max_msgs, aes_batch** out) {
  clear_error();
  if (!out) return set_error(AES_EINVAL, "null output pointer");
  *out = nullptr;
  if (!pool || !pool->entries) return set_error(AES_EINVAL, "null key pool");
  if (max_msgs == 0 || max_msgs > kMaxMsgs) return set_error(AES_EINVAL, "max_msgs must be 1..2^24 (got %zu)", max_msgs);
  aes_batch* b = new (std::nothrow) aes_batch();
  if (!b) return set_error(AES_ENOMEM, "host allocation failed");
  b->pool = pool;
  b->max_msgs = max_msgs;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) { delete b; return cuda_error(e, "cudaGetDevice"); }
  if (b->device != pool->device) { delete b; return set_error(AES_EINVAL, "pool and batch on different devices"); }
  const DeviceInfo* di = current_device_info();
  if (!di) { delete b; return AES_ECUDA; }
  b->wmax = size_t(di->sms) * (kMaxShapeThreads / 32);
  b->bytes = layout(max_msgs, max_msgs, b->wmax).end_iv;  // enough for any split of max_msgs, with IVs
  if ((e = cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    delete b;
    return cuda_error(e, "cudaStreamCreate");
  }
  for (Slot& s : b->slot) {
    if ((e = cudaMallocHost(&s.host, b->bytes)) != cudaSuccess || (e = cudaMalloc(&s.dev, b->bytes)) != cudaSuccess) {
      aes_batch_destroy(b);
      return set_error(AES_ENOMEM, "batch buffers (%zu bytes) could not be allocated: %s", b->bytes, cudaGetErrorString(e));
    }
    if ((e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming)) != cudaSuccess) {
      aes_batch_destroy(b);
      return cuda_error(e, "cudaEventCreate");
    }
  }
  *out = b;
  return AES_OK;
}

aes_status aes_batch_run(aes_batch* b, const aes_msg* msgs, size_t nmsgs, const void* d_in, void* d_out,
                         size_t buf_bytes, void* cuda_stream) {
  clear_error();
  if (!b) return set_error(AES_EINVAL, "null batch");
  std::lock_guard<std::mutex> lk(b->mu);
  return run_locked(b, msgs, nmsgs, d_in, d_out, buf_bytes, static_cast<cudaStream_t>(cuda_stream));
}

aes_status aes_batch_run_iv(aes_batch* b, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs, const void* d_in,
                            void* d_out, size_t buf_bytes, void* cuda_stream) {
  clear_error();
  if (!b) return set_error(AES_EINVAL, "null batch");
  std::lock_guard<std::mutex> lk(b->mu);
  return run_locked(b, msgs, nmsgs, d_in, d_out, buf_bytes, static_cast<cudaStream_t>(cuda_stream), ivs);
}

aes_status aes_batch_set_shape(aes_batch* b, int threads, int blocks_per_lane) {
  clear_error();
  if (!b) return set_error(AES_EINVAL, "null batch");
  if (!shape_compiled(threads, blocks_per_lane))
    return set_error(AES_EINVAL, "shape (%d threads, %d blocks per lane) is not compiled", threads, blocks_per_lane);
  std::lock_guard<std::mutex> lk(b->mu);
  b->threads = threads;
  b->bpl = blocks_per_lane;
  return AES_OK;
}

aes_status aes_batch_autotune(aes_batch* b, const aes_msg* msgs, size_t nmsgs, const void* d_in, void* d_out,
                              size_t buf_bytes, const char* cache_path, int* threads, int* blocks_per_lane,
                              void* cuda_stream) {
  clear_error();
  if (!b) return set_error(AES_EINVAL, "null batch");
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  std::lock_guard<std::mutex> lk(b->mu);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const std::string sig = signature(di, msgs, nmsgs);
  std::string text = cache_path ? read_file(cache_path) : std::string();
  int t = 0, u = 0;
  if (cache_path && cache_lookup(text, sig, &t, &u)) {
    b->threads = t;
    b->bpl = u;
  } else {
    cudaEvent_t e0, e1;
    cudaError_t ce;
    if ((ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess) return cuda_error(ce, "cudaEventCreate");
    double best = 1e30;
    Shape best_shape = kShapes[0];
    aes_status result = AES_OK;
    int nre = 0, nrd = 0;
    round_classes(b->pool, msgs, nmsgs, &nre, &nrd);
    for (const Shape& sh : kShapes) {
      if (!ttable_batched_dual(sh.threads, sh.bpl, nre, nrd)) continue;  // (768, 1) on other than AES-128
      b->threads = sh.threads;
      b->bpl = sh.bpl;
      if ((result = run_locked(b, msgs, nmsgs, d_in, d_out, buf_bytes, st)) != AES_OK) break;  // warm-up, builds the graph
      if ((result = run_locked(b, msgs, nmsgs, d_in, d_out, buf_bytes, st)) != AES_OK) break;  // graph for the other slot
      float ms_min = 1e30f;
      for (int rep = 0; rep < 3 && result == AES_OK; ++rep) {
        cudaEventRecord(e0, st);
        result = run_locked(b, msgs, nmsgs, d_in, d_out, buf_bytes, st);
        cudaEventRecord(e1, st);
        if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) { result = cuda_error(ce, "autotune timing"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      if (result != AES_OK) break;
      if (ms_min < best) { best = ms_min; best_shape = sh; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != AES_OK) return result;
    b->threads = best_shape.threads;
    b->bpl = best_shape.bpl;
    if (cache_path) cache_store(cache_path, text, sig, b->threads, b->bpl, best * 1e3);
  }
  if (threads) *threads = b->threads;
  if (blocks_per_lane) *blocks_per_lane = b->bpl;
  return AES_OK;
}

aes_status aes_crypt_batched_iv(aes_keypool* pool, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs,
                                const void* d_in, void* d_out, size_t buf_bytes, void* cuda_stream) {
  clear_error();
  if (!pool || !pool->entries || !pool->mu) return set_error(AES_EINVAL, "null key pool");
  std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(pool->mu));
  if (!pool->internal || pool->internal->max_msgs < nmsgs) {
    if (pool->internal) { aes_batch_destroy(pool->internal); pool->internal = nullptr; }
    aes_status st = aes_batch_create(pool, std::max<size_t>(nmsgs, 1024), &pool->internal);
    if (st != AES_OK) return st;
  }
  return aes_batch_run_iv(pool->internal, msgs, ivs, nmsgs, d_in, d_out, buf_bytes, cuda_stream);
}

aes_status aes_crypt_batched(aes_keypool* pool, const aes_msg* msgs, size_t nmsgs, const void* d_in,
                             void* d_out, size_t buf_bytes, void* cuda_stream) {
  return aes_crypt_batched_iv(pool, msgs, nullptr, nmsgs, d_in, d_out, buf_bytes, cuda_stream);
}

}  // extern "C"

extern "C" int aes_testing_weighted_slices(const uint64_t* nblocks, const int8_t* rounds, size_t n, uint64_t nw,
                                           uint64_t* gb, uint32_t* msg) {
  if (!nblocks || !rounds || !gb || !msg || n == 0 || n > (size_t(1) << 20) || nw == 0) return -1;
  std::vector<BatchMsg> m(n);
  std::vector<uint64_t> start(n + 1);
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    if (nblocks[i] == 0 || (rounds[i] != 10 && rounds[i] != 12 && rounds[i] != 14)) return -1;
    m[i] = BatchMsg{uint32_t(i), 0u, 0, 0, nblocks[i]};
    start[i] = total;
    total += nblocks[i];
  }
  start[n] = total;
  const uint64_t W = work_of(m.data(), n, rounds);
  weighted_slices(m.data(), start.data(), n, rounds, W, nw, gb, msg);
  return 0;
}
