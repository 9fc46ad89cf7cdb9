// pipe_rates.cu -- measures on one GPU the issue rates (lanes per SM-clock) of the integer
// instructions the on-chip AES roofline is built from: three-input logic (LOP3), adds, funnel
// shifts, byte permutes, integer multiply-adds, warp shuffles, byte-permute-addressed
// shared-memory lookups, and half-and-half mixes (to see whether two kinds issue side by side).
// A standalone measurement program for the test suite (tests/test_gpu_probes.py), not part of
// the library.
//
// One CTA of 1024 threads per SM (its dynamic shared memory leaves room for no second CTA),
// eight independent dependency chains per thread, 16 x 8 operations per loop trip; the cycle
// count of each CTA comes from clock64 between two barriers, so the rate does not depend on
// the clock frequency.  The operations are inline PTX, so the compiler cannot fold them.
// Prints one JSON object: {"<mix>": {"lanes_per_sm_clock": x, "implied_sm_mhz": f}, ...}.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

namespace {
__device__ __forceinline__ uint32_t p_lop3_96(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t p_lop3_e8(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t p_shf(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}
__device__ __forceinline__ uint32_t p_prmt(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}
__device__ __forceinline__ uint32_t p_add2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("{ .reg .u32 t; add.u32 t, %1, %2; add.u32 %0, t, %3; }" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t p_imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

constexpr int kProbeThreads = 1024;
constexpr int kProbeSmem = 160 * 1024;  // one CTA per SM
constexpr int kTableWords = 256 * 64;   // 64 KiB lookup table (entry x, lane l at word x*64 + l)

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1)
pipe_probe(uint32_t* out, long long* cyc, uint32_t b, uint32_t c, int iters) {
  extern __shared__ uint32_t tbl[];
  const int tid = threadIdx.x;
  const uint32_t lanec = (tid & 31) * 4u;
  if (OP == 6)
    for (int i = tid; i < kTableWords; i += blockDim.x) tbl[i] = (uint32_t(i) * 2654435761u) ^ uint32_t(i >> 3);
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = uint32_t(tid * 8 + i) * 0x9E3779B9u + b;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (OP == 0) a[i] = (u & 1) ? p_lop3_e8(a[i], a[(i + 1) & 7], b) : p_lop3_96(a[i], a[(i + 3) & 7], c);
        if (OP == 1) a[i] = p_add2(a[i], a[(i + 1) & 7], b);
        if (OP == 2) a[i] = p_shf(a[i], a[(i + 1) & 7], b + u);
        if (OP == 3) a[i] = p_prmt(a[i], a[(i + 1) & 7], (u & 1) ? 0x5140u : 0x3726u);
        if (OP == 4) a[i] = p_imad(a[i], a[(i + 1) & 7] | 1u, b);
        if (OP == 5) a[i] = __shfl_xor_sync(0xFFFFFFFFu, a[i], ((i + u) & 31) | 1) + a[i];
        if (OP == 6) {
          // byte (u mod 4) of a[i] -> byte 1, 4 * lane -> byte 0: a word offset below 256 * 64
          const uint32_t addr = p_prmt(a[i], lanec, 0x5504u + ((u & 3) << 4));
          a[i] ^= tbl[addr >> 2];
        }
        if (OP == 7) a[i] = (i & 1) ? p_imad(a[i], a[(i + 1) & 7] | 1u, b) : p_lop3_96(a[i], a[(i + 3) & 7], c);
        if (OP == 8) a[i] = (i & 1) ? p_shf(a[i], a[(i + 1) & 7], b + u) : p_lop3_96(a[i], a[(i + 3) & 7], c);
        if (OP == 9) a[i] = (i & 1) ? p_prmt(a[i], a[(i + 1) & 7], 0x5140u) : p_lop3_96(a[i], a[(i + 3) & 7], c);
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (tid == 0) cyc[blockIdx.x] = t1 - t0;
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r ^= a[i];
  out[size_t(blockIdx.x) * blockDim.x + tid] = r;  // keeps the chains live
}

using ProbeFn = void (*)(uint32_t*, long long*, uint32_t, uint32_t, int);

ProbeFn probe_kernel(int op) {
  switch (op) {
    case 0: return pipe_probe<0>;
    case 1: return pipe_probe<1>;
    case 2: return pipe_probe<2>;
    case 3: return pipe_probe<3>;
    case 4: return pipe_probe<4>;
    case 5: return pipe_probe<5>;
    case 6: return pipe_probe<6>;
    case 7: return pipe_probe<7>;
    case 8: return pipe_probe<8>;
    case 9: return pipe_probe<9>;
    default: return nullptr;
  }
}

}  // namespace

// Rate of one mix: 0 on success.
static int pipe_rate(int op, int iters, double* lanes_per_clk, double* implied_mhz) {
  ProbeFn k = probe_kernel(op);
  if (!k || iters < 1 || iters > (1 << 16)) return -1;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || nsm <= 0) return -1;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem) !=
      cudaSuccess)
    return -1;
  uint32_t* d_out = nullptr;
  long long* d_cyc = nullptr;
  if (cudaMalloc(&d_out, sizeof(uint32_t) * size_t(nsm) * kProbeThreads) != cudaSuccess) return -1;
  if (cudaMalloc(&d_cyc, sizeof(long long) * size_t(nsm)) != cudaSuccess) {
    cudaFree(d_out);
    return -1;
  }
  int rc = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  std::vector<long long> h(size_t(nsm), 0);
  k<<<nsm, kProbeThreads, kProbeSmem>>>(d_out, d_cyc, 0x12345678u, 0x0F0F1234u, 16);  // warm-up
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = -1;
  if (rc == 0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = -1;
  if (rc == 0) {
    cudaEventRecord(e0);
    k<<<nsm, kProbeThreads, kProbeSmem>>>(d_out, d_cyc, 0x12345678u, 0x0F0F1234u, iters);
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) rc = -1;
  }
  if (rc == 0 && (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                  cudaMemcpy(h.data(), d_cyc, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = -1;
  if (rc == 0) {
    double sum = 0;
    for (long long v : h) sum += double(v);
    const double cycles = sum / nsm;  // per CTA
    const double ops = double(kProbeThreads) * iters * 16 * 8;
    *lanes_per_clk = ops / cycles;
    *implied_mhz = ms > 0 ? cycles / (double(ms) * 1e3) : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  cudaFree(d_cyc);
  return rc;
}

int main() {
  static const char* names[] = {"lop3", "iadd", "shf", "prmt", "imad", "shfl (+ add)",
                                "prmt-addressed lds.32 lookup (+ xor)", "imad | lop3 50/50", "shf | lop3 50/50",
                                "prmt | lop3 50/50"};
  int sms = 0, mhz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&mhz, cudaDevAttrClockRate, 0);
  std::printf("{\"sms\": %d, \"clock_khz\": %d", sms, mhz);
  for (int op = 0; op < 10; ++op) {
    double lanes = 0, implied = 0;
    if (pipe_rate(op, 4096, &lanes, &implied) != 0) {
      std::fprintf(stderr, "pipe probe %s failed\n", names[op]);
      return 1;
    }
    std::printf(", \"%s\": {\"lanes_per_sm_clock\": %.2f, \"implied_sm_mhz\": %.0f}", names[op], lanes, implied);
  }
  std::printf("}\n");
  return 0;
}
