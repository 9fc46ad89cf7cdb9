// aes_internal.cuh -- declarations shared by the library's translation units (not part of
// the C ABI; include/aesgb.h is the public surface).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>

#include "aes_field.cuh"
#include "aesgb.h"

namespace aesgb {

constexpr int kMaxRounds = 14;

// Round keys as little-endian column words, passed by value as a kernel parameter so that
// every AddRoundKey reads its operand from the constant bank (no memory traffic per block).
struct KeyWords {
  uint32_t w[kMaxRounds + 1][4];
};


// ---- errors -------------------------------------------------------------------------
aes_status set_error(aes_status st, const char* fmt, ...);
aes_status cuda_error(cudaError_t e, const char* what);
void clear_error();

// ---- device facts ---------------------------------------------------------------------
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;  // max dynamic shared memory per block (bytes)
  // kernels may load and store any host memory (pageable access through the host's page
  // tables, as on Grace-Blackwell over NVLink-C2C)
  bool host_direct = false;
  char name[256] = {0};
};
// Info for the current device (cached per device).  Returns nullptr and sets the error on
// a CUDA failure.
const DeviceInfo* current_device_info();

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current device, once per
// (device, kernel, size): later calls find it in a small cache and skip the driver call, which
// would otherwise sit on every launch's critical path.
aes_status ensure_kernel_smem(const void* fn, size_t bytes);
// Resident CTAs per SM of a kernel on the current device (cached like ensure_kernel_smem).
aes_status kernel_ctas_per_sm(const void* fn, int threads, size_t smem, int* out);

// ---- key words -------------------------------------------------------------------------
// Encryption: round key 0 has the IV folded in (C = E(P ^ IV) needs P ^ IV ^ K0).
KeyWords enc_key_words(const aes_key_schedule& ks, const uint8_t* iv);
// Decryption, equivalent inverse cipher: word r is InvMixColumns(K[nr - r]) for
// 0 < r < nr, K[nr] first, K[0] ^ IV last (P = D(C) ^ IV).
KeyWords dec_key_words(const aes_key_schedule& ks, const uint8_t* iv);
bool schedule_ok(const aes_key_schedule* ks);

// ---- launch configurations --------------------------------------------------------------
struct TTConfig {
  int threads = 512;  // CTA size (see tt::select_config for the compiled pairs)
  int unroll = 2;     // blocks per thread in flight
  int ctas_per_sm = 1;
};

struct BSConfig {
  int reserved = 0;  // one compiled shape: 128-thread CTAs, 32 blocks per thread
};

using TTKernelFn = void (*)(const uint4*, uint4*, size_t, const KeyWords);
TTKernelFn ttable_kernel_r10(int dir, int threads, int unroll);
TTKernelFn ttable_kernel_r12(int dir, int threads, int unroll);
TTKernelFn ttable_kernel_r14(int dir, int threads, int unroll);

aes_status launch_ttable(int dir, int nr, const KeyWords& kw, const void* d_in, void* d_out,
                         size_t nblocks, cudaStream_t stream, const TTConfig& cfg);
// The bitsliced kernels take the plain schedule (they run the paper's inverse-cipher order,
// not the equivalent inverse cipher); the IV is folded into round key 0.
// The tuned choice for AES_IMPL_AUTO on the current device (aes_autotune_blocks); false when
// none was tuned (then the default T-table shape is used).  *pinned (if not null) tells whether
// the choice was set by aes_set_auto_choice, which serves calls of every size.
bool tuned_choice(int dir, int nr, int* impl, TTConfig* cfg, bool* pinned = nullptr);
// AES_IMPL_AUTO calls of at most this many blocks (and no pinned choice) take the small-call
// kernel, whose tables need no shared-memory fill (aes_small.cu).
constexpr size_t kSmallCallBlocks = 32768;
aes_status launch_small(int dir, int nr, const KeyWords& kw, const void* d_in, void* d_out, size_t nblocks,
                        cudaStream_t stream);
aes_status launch_bitslice(int dir, const aes_key_schedule& ks, const uint8_t* iv, const void* d_in,
                           void* d_out, size_t nblocks, cudaStream_t stream, const BSConfig& cfg);

// Shared-memory bytes one T-table CTA needs for direction `dir`.
size_t ttable_smem_bytes(int dir);

// Launch shape of a four-lanes-per-chain CBC encryption (tt::col_round) over `chains` chains:
// CTA threads (at least 128, so that the table fill is quick), the warps of a CTA that run
// chains (the others only help fill the tables), grid, and chains per warp (lanes 4 cpw .. 31
// of each chain warp idle).
struct ColsShape {
  unsigned threads, wpc, grid, cpw;
};
ColsShape cols_shape(uint64_t chains, int sms);

// ---- key pool ------------------------------------------------------------------------------
// One device-resident key: the encryption words and the equivalent-inverse-cipher words
// (InvMixColumns applied to the middle round keys), both in round order.  512 bytes.
struct PoolEntry {
  uint32_t enc[kMaxRounds + 1][4];
  uint32_t dec[kMaxRounds + 1][4];
  int32_t nr;
  uint32_t pad[7];
};
static_assert(sizeof(PoolEntry) == 512, "pool entries are 512 bytes");

// ---- batched messages ------------------------------------------------------------------------
struct BatchMsg {
  uint32_t key_idx;
  uint32_t pad;
  uint64_t src_block;  // first input block, counted from the input base address
  uint64_t dst_block;  // first output block, counted from the output base address
  uint64_t nblocks;
};
static_assert(sizeof(BatchMsg) == 32, "batch descriptors are 32 bytes");

// Work of one direction: messages laid end to end; start[m] is the first block of message m
// in that virtual block space (nmsgs + 1 entries, the last = total).
// warp_msg[w] (optional, may be null) is the message holding warp w's first block when the
// kernel runs with exactly the warps the table was made for; warp_gb (optional, nwarps + 1
// entries) gives each warp's first block, so that the host can balance the slices by work
// (blocks x rounds) rather than by blocks.  Without it every warp takes an equal block range.
// ivs (optional, nmsgs entries): message m's IV, XORed into every block of m before the
// cipher (encryption) or after the inverse cipher (decryption); null means zero IVs.
struct BatchDir {
  const BatchMsg* msgs;
  const uint64_t* start;
  const uint32_t* warp_msg;
  uint64_t total;
  uint32_t nmsgs;
  uint32_t pad;
  const uint64_t* warp_gb;
  const uint4* ivs;
};

// Kernel arguments: input and output base addresses as integers (the server passes 0 and
// absolute block numbers), the direction's work, the key pool.
using TTBatchedFn = void (*)(uint64_t, uint64_t, const BatchDir, const PoolEntry*);
// Both directions in one launch: the first `ge` CTAs encrypt, the rest decrypt.
using TTDualFn = void (*)(uint64_t, uint64_t, const BatchDir, const BatchDir, const PoolEntry*, uint32_t);
// Compiled shapes (CTA threads, blocks per lane per window) for nre / nrd, the round count
// of every encryption / decryption message (0 when mixed); the kernel specialised to those
// counts where one is compiled, else the generic one; nullptr if the shape is not compiled
// for them.
TTDualFn ttable_batched_dual(int threads, int blocks_per_lane, int nre, int nrd);
TTDualFn ttable_batched_dual_wide(int threads, int blocks_per_lane);  // the U = 4 shapes
TTDualFn ttable_batched_dual_r10(int threads, int blocks_per_lane, int nre, int nrd);  // AES-128 only

}  // namespace aesgb

struct aes_batch;

namespace aesgb {
// A handful of messages launched with their descriptors as kernel parameters (no upload, no
// graph, no shared-memory tables): the request server's path for small batches (aes_small.cu).
constexpr int kSmallBatchMax = 16;
struct SmallMsg {
  uint64_t src, dst;  // byte addresses, 16-byte aligned
  uint32_t nblocks, key_idx, dir, pad;
};
struct SmallBatch {
  uint32_t n, pad;
  uint64_t start[kSmallBatchMax + 1];  // first block of each message in the batch's block space
  SmallMsg m[kSmallBatchMax];
};
aes_status launch_small_batch(const SmallBatch& b, const PoolEntry* pool, cudaStream_t stream);

// Work of a direction in round-blocks: sum of nblocks x rounds[key_idx] over its messages.
uint64_t work_of(const BatchMsg* m, size_t n, const int8_t* rounds);
// Cuts a direction's block space (n messages, start[0..n]) into nw slices of equal work W in
// round-blocks: gb[w] is warp w's first block (gb[nw] = start[n]) and msg[w] the message
// holding it.
void weighted_slices(const BatchMsg* m, const uint64_t* start, size_t n, const int8_t* rounds, uint64_t W,
                     uint64_t nw, uint64_t* gb, uint32_t* msg);
// Launches one batch from descriptors written by `fill(enc, dec, enc_ivs, dec_ivs)` (nenc and
// ndec entries, nblocks > 0 each) relative to in_base / out_base; with with_ivs the fill also
// writes one IV per descriptor (in the same order), else the IV pointers are null.  The
// caller holds the batch's lock.
using DescFill = std::function<void(BatchMsg*, BatchMsg*, uint4*, uint4*)>;
aes_status batch_launch_descs(aes_batch* b, size_t nenc, size_t ndec, const DescFill& fill, bool with_ivs,
                              uint64_t in_base, uint64_t out_base, cudaStream_t stream);
}  // namespace aesgb

struct aes_keypool {
  int device = -1;
  size_t capacity = 0;
  aesgb::PoolEntry* entries = nullptr;  // device
  uint8_t* raw = nullptr;               // device staging for raw keys
  size_t raw_cap = 0;                   // bytes
  int8_t* nr = nullptr;                 // host shadow: rounds per slot (0 = empty)
  aes_batch* internal = nullptr;        // for aes_crypt_batched
  void* mu = nullptr;                   // std::mutex*, serialises aes_crypt_batched and aes_cbc_batched
  void* cbc = nullptr;                  // descriptor buffers of aes_cbc_batched (aes_cbc_batched.cu)
};

namespace aesgb {
// Frees the pool's aes_cbc_batched buffers (called by aes_keypool_destroy).
void cbc_batched_release(aes_keypool* pool);
}  // namespace aesgb
