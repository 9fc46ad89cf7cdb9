// aes_ttable.cu -- host launcher for the T-table kernels (kernels: aes_ttable.cuh,
// instantiated per round count in aes_ttable_r{10,12,14}.cu).
#include "aes_internal.cuh"

namespace aesgb {

namespace {
constexpr uint32_t kRegionBytes = 65536;
}

size_t ttable_smem_bytes(int dir) { return (dir == AES_ENCRYPT ? 2 : 3) * size_t(kRegionBytes); }

aes_status launch_ttable(int dir, int nr, const KeyWords& kw, const void* d_in, void* d_out,
                         size_t nblocks, cudaStream_t stream, const TTConfig& cfg) {
  TTKernelFn k = nr == 10 ? ttable_kernel_r10(dir, cfg.threads, cfg.unroll)
                 : nr == 12 ? ttable_kernel_r12(dir, cfg.threads, cfg.unroll)
                 : nr == 14 ? ttable_kernel_r14(dir, cfg.threads, cfg.unroll)
                            : nullptr;
  if (!k) return set_error(AES_EINVAL, "no T-table kernel for nr=%d threads=%d unroll=%d", nr, cfg.threads, cfg.unroll);
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  const size_t smem = ttable_smem_bytes(dir);
  if (smem > size_t(di->smem_optin))
    return set_error(AES_EINVAL, "device allows %d bytes of shared memory per block, T-tables need %zu",
                     di->smem_optin, smem);
  aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(k), smem);
  if (ast != AES_OK) return ast;
  cudaError_t e;
  const size_t want = (nblocks + cfg.threads - 1) / cfg.threads;
  const size_t cap = size_t(di->sms) * size_t(cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : 1);
  const unsigned grid = unsigned(want < cap ? want : cap);
  k<<<grid, cfg.threads, smem, stream>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out),
                                          nblocks, kw);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "T-table kernel launch");
  return AES_OK;
}

}  // namespace aesgb
