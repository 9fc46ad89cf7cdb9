/*
 * aesgb.h -- C ABI of the GB300 AES library (libaesgb.so).
 *
 * The library computes the paper's cipher (Kepner et al., "Parallel Vectorized Algebraic
 * AES in MATLAB ...", arXiv:1506.08503): AES built from GF(2^8) arithmetic (Section II),
 * applied to many independent 16-byte blocks at once (the paper's vectorisation over N
 * messages, Section II and Section III).  Each block is one message of the paper's CBC
 * mode: C = Cipher_K(P xor IV) and P = InvCipher_K(C) xor IV (App. A1 and A4 with one
 * block per message).  IV = NULL gives plain ECB.
 *
 * Conventions for every entry point:
 *  - Every function returns an aes_status; none aborts, throws or exits.  On failure
 *    aes_last_error() returns a message for the calling thread.
 *  - "Device pointer" means memory the CUDA device can address (cudaMalloc, torch tensor
 *    storage), caller-owned, 16-byte aligned unless stated.  "Host pointer" means ordinary
 *    host memory, caller-owned.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Work is enqueued asynchronously; errors raised by a kernel surface at the next
 *    synchronisation of that stream.
 *  - A block is 16 bytes in the paper's column-major state order: byte i is row i % 4,
 *    column i / 4 (App. A1's ShiftRows indices).  Buffers hold whole blocks: padding to a
 *    block boundary is the caller's job (the paper zero-pads, App. A1).
 */
#ifndef AESGB_H
#define AESGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int aes_status;
#define AES_OK 0
#define AES_EINVAL (-1)    /* bad argument: size, alignment, overlap, key length, index */
#define AES_ENOMEM (-2)    /* a device or host allocation failed, or a budget is exceeded */
#define AES_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define AES_EAGAIN (-4)    /* a queue is full; retry later */
#define AES_ETIMEDOUT (-5) /* a bounded wait ran out */
#define AES_ENOTFOUND (-6) /* unknown ticket or handle */

/* Direction of a request. */
#define AES_ENCRYPT 0
#define AES_DECRYPT 1

/* Kernel family.  AUTO picks the fastest for the device (the T-table kernel on GB300);
 * BITSLICE is the constant-time circuit, whose memory accesses do not depend on data or key. */
#define AES_IMPL_AUTO 0
#define AES_IMPL_TTABLE 1
#define AES_IMPL_BITSLICE 2

/* Message for the last error on the calling thread ("" if none).  The pointer stays valid
 * until the next library call on this thread. */
const char* aes_last_error(void);

/* Version string, e.g. "aesgb 1.0 sm_103a". */
const char* aes_version(void);

/* ---------------------------------------------------------------------------------------
 * Key schedule (App. A3 for 128-bit keys; the 192/256-bit schedules follow the AES
 * standard's general Nk-word rule, FIPS-197 Section 5.2, since the paper treats 128 bits).
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int32_t nr;            /* number of rounds: 10, 12 or 14 */
  uint8_t rk[15][16];    /* round keys 0..nr in block byte order; rows > nr are zero */
} aes_key_schedule;

/* Expands `key` (host pointer, key_bits/8 bytes) into `out` (host, caller-owned).
 * key_bits must be 128, 192 or 256, else AES_EINVAL.  Runs on the host; no CUDA call. */
aes_status aes_key_expand(const uint8_t* key, int key_bits, aes_key_schedule* out);

/* ---------------------------------------------------------------------------------------
 * Many independent blocks under one key (the paper's N x 16 matrix, Section II).
 *   ks        host pointer to an expanded schedule (copied into the launch; may be freed
 *             as soon as the call returns)
 *   iv        host pointer to 16 bytes, or NULL for a zero IV (ECB); folded into the round
 *             keys, so it costs nothing per block
 *   d_in      device pointer, nblocks * 16 bytes, 16-byte aligned
 *   d_out     device pointer, same size and alignment; d_out == d_in (in place) is allowed,
 *             any other overlap is AES_EINVAL
 *   nblocks   number of 16-byte blocks; 0 returns AES_OK without a launch
 * Returns AES_EINVAL for a bad pointer/size/schedule, AES_ECUDA if the launch fails.
 * ------------------------------------------------------------------------------------- */
aes_status aes_encrypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                              void* d_out, size_t nblocks, void* cuda_stream);
aes_status aes_decrypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                              void* d_out, size_t nblocks, void* cuda_stream);

/* Same, with the direction (AES_ENCRYPT / AES_DECRYPT) and kernel family (AES_IMPL_*)
 * chosen explicitly.  An unknown dir or impl is AES_EINVAL. */
aes_status aes_crypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                            void* d_out, size_t nblocks, int dir, int impl, void* cuda_stream);

/* Same cipher on HOST buffers: the library copies the data to the device in 64 MiB chunks,
 * runs the kernel and copies the result back, overlapping the three on its own streams.
 *   h_in, h_out  host pointers (pinned memory gives full copy bandwidth; pageable works,
 *                slower), nblocks * 16 bytes, no alignment rule; in place allowed
 *   cuda_stream  the copies start after the work already queued on this stream
 * Blocks until h_out holds the result.  The first call on a device allocates the staging
 * buffers (3 x 64 MiB, kept until process exit); AES_ENOMEM if that fails.  Calls on one
 * device are serialised. */
aes_status aes_crypt_host(const aes_key_schedule* ks, const uint8_t* iv, const void* h_in, void* h_out,
                          size_t nblocks, int dir, int impl, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AESGB_H */
