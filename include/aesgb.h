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
 * chosen explicitly.  An unknown dir or impl is AES_EINVAL.  AES_IMPL_AUTO takes the choice
 * aes_autotune_blocks made for this device, direction and round count, else the T-tables
 * with 512-thread CTAs and two blocks in flight per thread; calls of at most 32768 blocks
 * take a T-table kernel that reads its tables from global memory through the read-only cache
 * (no per-CTA fill of shared-memory tables: a small call's latency), unless
 * aes_set_auto_choice has pinned the choice. */
aes_status aes_crypt_blocks(const aes_key_schedule* ks, const uint8_t* iv, const void* d_in,
                            void* d_out, size_t nblocks, int dir, int impl, void* cuda_stream);

/* Tunes AES_IMPL_AUTO for the current device, `dir` and ks->nr: times every compiled
 * candidate on d_in -> d_out (nblocks blocks, device, 16-byte aligned; d_out is overwritten):
 * the T-table kernel with CTAs of 512 threads and 1, 2 or 4 blocks in flight per thread, 256
 * threads and 4, 768 threads and 2, 1024 threads and 1 or 2, and the bitsliced kernel (32
 * blocks per thread).
 * The fastest serves later AES_IMPL_AUTO calls in this process.  If cache_path is not NULL
 * the choice is also recorded in that JSON file, keyed by device name, direction, round count
 * and floor(log2(nblocks)); an existing entry is used without timing.  Writes the choice to
 * *impl (AES_IMPL_TTABLE or AES_IMPL_BITSLICE), *threads and *unroll when not NULL.
 * Synchronous: it waits for its timing launches.  nblocks = 0 is AES_EINVAL. */
aes_status aes_autotune_blocks(const aes_key_schedule* ks, const void* d_in, void* d_out, size_t nblocks, int dir,
                               const char* cache_path, int* impl, int* threads, int* unroll, void* cuda_stream);

/* Sets the AES_IMPL_AUTO choice for the current device, `dir` and round count `nr` (10, 12,
 * 14) directly, without timing: impl AES_IMPL_TTABLE with one of the (threads, unroll) pairs
 * aes_autotune_blocks tries, or AES_IMPL_BITSLICE with (128, 32).  AES_EINVAL otherwise.  The
 * choice is pinned: it serves AES_IMPL_AUTO calls of every size, small calls included.
 * impl = AES_IMPL_AUTO (threads and unroll ignored) clears the tuned or pinned choice, back to
 * the default. */
aes_status aes_set_auto_choice(int dir, int nr, int impl, int threads, int unroll);

/* The paper's CBC mode over whole messages (Section II; App. A1 encryption, App. A4
 * decryption).  d_in and d_out (device) hold an nmsgs x (16 * blocks_per_msg) byte matrix, one
 * message per row, rows back to back; row i is chained: C_j = E(P_j xor C_{j-1}) with
 * C_{-1} = IV_i, and P_j = D(C_j) xor C_{j-1}.  d_ivs (device, 16-byte aligned) holds one
 * 16-byte IV for every row (iv_per_msg = 0, the appendix's repeated IV) or one per row
 * (iv_per_msg = 1, the IV matrix V of Section II).  Encryption is serial inside a message:
 * up to 64 messages per SM run four lanes to a message (one per state column), more run one
 * lane per message; decryption runs one lane per block.  Encryption may run in
 * place; decryption may not (each block needs the previous ciphertext): AES_EINVAL.  An empty
 * matrix returns AES_OK. */
aes_status aes_cbc_crypt(const aes_key_schedule* ks, const void* d_ivs, int iv_per_msg, const void* d_in,
                         void* d_out, size_t nmsgs, size_t blocks_per_msg, int dir, void* cuda_stream);

/* Counter mode, a follow-on the paper names as future work (Section V): block i becomes
 * in_i xor Cipher(T + i), where T is the 16-byte initial counter block ctr0 (host pointer)
 * read as a big-endian 128-bit integer and the sum is taken mod 2^128.  Encryption and
 * decryption are the same call.  Buffer rules as aes_crypt_blocks (device, 16-byte aligned,
 * in place allowed). */
aes_status aes_ctr_crypt(const aes_key_schedule* ks, const uint8_t* ctr0, const void* d_in, void* d_out,
                         size_t nblocks, void* cuda_stream);

/* AES-GCM, the counter-based authenticated mode that Section V of the paper names as future
 * work; the paper does not define it, so this follows NIST SP 800-38D.  J0 = IV || 0^31 || 1
 * for a 96-bit IV, else GHASH_H of the IV zero-padded to whole blocks and a block holding its
 * 64-bit bit length (computed in the kernel).  Data block j is XORed with Cipher(J0 with its
 * last 32 bits, big-endian, increased by 1 + j mod 2^32), and the 16-byte tag is Cipher(J0) +
 * GHASH_H over the AAD and the ciphertext (each zero-padded to whole blocks) and the two bit
 * lengths, H = Cipher(0).
 *   ks         any schedule from aes_key_expand (AES-128/192/256)
 *   iv, iv_len host IV of 1 to 256 bytes (12 is the recommended length); else AES_EINVAL
 *   d_aad      device, aad_len bytes (any length up to 64 GiB, 16-byte aligned pointer),
 *              authenticated, not encrypted; may be NULL when aad_len is 0
 *   d_in/d_out device, nbytes bytes (any length up to (2^32 - 2) * 16), 16-byte aligned;
 *              in place allowed, partial overlap is AES_EINVAL; d_out must not overlap d_aad
 *   dir        AES_ENCRYPT hashes the output, AES_DECRYPT hashes the input (the ciphertext)
 *   d_tag      device, 16 bytes, any alignment: receives the tag.  On decryption it is the
 *              tag computed from the ciphertext: the caller compares it with the received tag
 *              before trusting the plaintext
 *   d_work     device workspace of at least aes_gcm_workspace_bytes() bytes (a few KiB: one
 *              partial sum per CTA and a ticket), 16-byte aligned, owned by the caller; calls
 *              that share a workspace must be ordered on one stream, and it must not overlap
 *              any other buffer
 * One kernel launch on cuda_stream (after a 4-byte memset of the ticket); asynchronous. */
size_t aes_gcm_workspace_bytes(void);
aes_status aes_gcm_crypt(const aes_key_schedule* ks, const uint8_t* iv, size_t iv_len, const void* d_aad,
                         size_t aad_len, const void* d_in, void* d_out, size_t nbytes, int dir, uint8_t* d_tag,
                         void* d_work, size_t work_bytes, void* cuda_stream);

/* AES-GCM decryption with the tag check on the device: aes_gcm_crypt with dir = AES_DECRYPT
 * (same arguments and rules), and *d_ok (device int, int-aligned) receives 1 when the tag
 * computed from the ciphertext equals the 16 bytes at d_expected_tag (device, any alignment),
 * else 0; all 16 bytes are compared, with no early exit.  The plaintext is written either way:
 * use it only when *d_ok is 1.  d_expected_tag and d_ok must not overlap d_out, d_tag, the
 * workspace or each other; NULL for either is AES_EINVAL.  Same single launch. */
aes_status aes_gcm_decrypt_verify(const aes_key_schedule* ks, const uint8_t* iv, size_t iv_len, const void* d_aad,
                                  size_t aad_len, const void* d_in, void* d_out, size_t nbytes,
                                  const uint8_t* d_expected_tag, int* d_ok, uint8_t* d_tag, void* d_work,
                                  size_t work_bytes, void* cuda_stream);

/* Equality query on a deterministically encrypted column (the encrypted-database use the
 * paper motivates in Section I): under one key and IV, equal 16-byte records have equal
 * ciphertexts, so the records equal to a query are those whose ciphertext equals the query's
 * ciphertext `needle` (16 bytes, host).  Scans d_column (device, nrecords x 16 bytes, 16-byte
 * aligned), writes the total number of matches to *d_count (device uint64, zeroed by the call)
 * and the first min(count, max_matches) matching record indices to d_matches (device uint64,
 * in no particular order).  Asynchronous on cuda_stream. */
aes_status aes_scan_equal(const void* d_column, size_t nrecords, const uint8_t* needle, uint64_t* d_matches,
                          size_t max_matches, uint64_t* d_count, void* cuda_stream);

/* Same cipher on HOST buffers.  On a device whose kernels may access host memory directly
 * (pageable access through the host page tables, e.g. Grace-Blackwell over NVLink-C2C) and
 * with both buffers 16-byte aligned, the kernel reads h_in and writes h_out itself, on
 * cuda_stream.  Otherwise the library copies the data to the device in 64 MiB chunks, runs
 * the kernel and copies the result back, overlapping the three on its own streams.
 *   h_in, h_out  host pointers (pinned memory gives full copy bandwidth; pageable works,
 *                slower, on the copy path), nblocks * 16 bytes; in place allowed
 *   cuda_stream  the work starts after the work already queued on this stream
 * Blocks until h_out holds the result.  The first copy-path call on a device allocates the
 * staging buffers (3 x 64 MiB, kept until process exit); AES_ENOMEM if that fails.  Copy-path
 * calls on one device are serialised. */
aes_status aes_crypt_host(const aes_key_schedule* ks, const uint8_t* iv, const void* h_in, void* h_out,
                          size_t nblocks, int dir, int impl, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Key pool: expanded schedules resident in device memory, addressed by index.  The paper's
 * key tensor K (R x N x 16, Section II) with one schedule per message.
 * ------------------------------------------------------------------------------------- */
typedef struct aes_keypool aes_keypool;

/* Allocates device memory for `capacity` schedules (512 bytes each) on the current device.
 * capacity must be 1..2^24, else AES_EINVAL; AES_ENOMEM if the allocation fails.  The pool
 * is owned by the library until aes_keypool_destroy. */
aes_status aes_keypool_create(size_t capacity, aes_keypool** out);

/* Expands `count` raw keys (host pointer, count * key_bits/8 bytes, back to back) ON THE
 * DEVICE into slots first .. first+count-1, together with their equivalent-inverse-cipher
 * schedules for decryption.  key_bits: 128, 192 or 256.  Returns once the schedules are
 * resident (it synchronises `cuda_stream`).  Slots out of range are AES_EINVAL. */
aes_status aes_keypool_load_keys(aes_keypool* pool, uint32_t first, size_t count, const uint8_t* keys,
                                 int key_bits, void* cuda_stream);

/* Copies one host-expanded schedule into slot `idx` (synchronous). */
aes_status aes_keypool_set(aes_keypool* pool, uint32_t idx, const aes_key_schedule* ks);

/* Number of rounds of slot idx (10, 12 or 14), or 0 if the slot was never loaded. */
int aes_keypool_rounds(const aes_keypool* pool, uint32_t idx);

/* Frees the pool's device memory.  NULL is a no-op.  The caller must not destroy a pool
 * while work that uses it is still queued. */
aes_status aes_keypool_destroy(aes_keypool* pool);

/* ---------------------------------------------------------------------------------------
 * Batched messages: many messages, each with its own key slot, direction and length, in one
 * persistent launch per direction (replayed from a CUDA graph).  Blocks of a message are
 * independent (the paper's one-block CBC messages, i.e. ECB under that message's key).
 * ------------------------------------------------------------------------------------- */
typedef struct {
  uint32_t key_idx; /* slot in the key pool (must be loaded) */
  uint32_t dir;     /* AES_ENCRYPT or AES_DECRYPT */
  uint64_t offset;  /* byte offset into both buffers, a multiple of 16 */
  uint64_t length;  /* bytes, a multiple of 16 (0 allowed: nothing to do) */
} aes_msg;

typedef struct aes_batch aes_batch;

/* A reusable batch context bound to `pool`: device descriptor buffers, pinned staging and the
 * cached CUDA graph.  max_msgs is the largest message count a single run may carry
 * (1..2^24).  Its launch shape starts at 768-thread CTAs with 1 block per lane per window,
 * which runs launches whose messages all use AES-128 keys and takes 512-thread CTAs for any
 * other (see aes_batch_autotune).  AES_ENOMEM if its buffers cannot be allocated. */
aes_status aes_batch_create(aes_keypool* pool, size_t max_msgs, aes_batch** out);

/* Runs every message of `msgs` (host array of nmsgs <= max_msgs) reading d_in and writing
 * d_out (device pointers, each buf_bytes long, 16-byte aligned; d_in == d_out allowed).
 * Asynchronous on cuda_stream; the host array may be reused as soon as the call returns.
 * A message whose [offset, offset+length) leaves the buffers, a length or offset that is not
 * a multiple of 16, an unloaded key slot or a bad dir is AES_EINVAL (nothing launched). */
aes_status aes_batch_run(aes_batch* b, const aes_msg* msgs, size_t nmsgs, const void* d_in, void* d_out,
                         size_t buf_bytes, void* cuda_stream);

/* aes_batch_run with one IV per message, the IV matrix V of the paper's Section II (one row
 * per message): ivs is a host array of nmsgs x 16 bytes (row i belongs to msgs[i]; NULL is
 * the same as aes_batch_run, zero IVs).  Every block of message i is one of the paper's
 * one-block CBC messages under that message's key and IV: C = Cipher_K(P xor IV_i) for
 * encryption, P = InvCipher_K(C) xor IV_i for decryption.  The IV is folded into the round key
 * that carries it when a warp moves to the message, so it costs nothing per block.  The array
 * is copied before the call returns.  Other rules as aes_batch_run. */
aes_status aes_batch_run_iv(aes_batch* b, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs, const void* d_in,
                            void* d_out, size_t buf_bytes, void* cuda_stream);

/* Tunes the batch's launch shape on this workload: the CTA size and the blocks each lane
 * enciphers per window; compiled pairs are (512, 1), (512, 2), (512, 4), (384, 4), (256, 4)
 * and, for work that is AES-128 throughout, (768, 1), one CTA per SM.  A direction whose
 * messages all use AES-128 keys runs a kernel specialised to 10 rounds.  It
 * times every candidate compiled for `msgs` (it overwrites d_out), keeps the fastest and, if
 * cache_path is not NULL, records it in that JSON file keyed by device name and workload
 * signature (an existing entry is reused without timing).  Writes the chosen shape to
 * *threads and *blocks_per_lane when they are not NULL. */
aes_status aes_batch_autotune(aes_batch* b, const aes_msg* msgs, size_t nmsgs, const void* d_in, void* d_out,
                              size_t buf_bytes, const char* cache_path, int* threads, int* blocks_per_lane,
                              void* cuda_stream);

/* Sets the launch shape directly (see aes_batch_autotune for the meaning); AES_EINVAL for a
 * shape that is not compiled. */
aes_status aes_batch_set_shape(aes_batch* b, int threads, int blocks_per_lane);

aes_status aes_batch_destroy(aes_batch* b);

/* One-shot form of aes_batch_run through a batch context the pool keeps internally (created
 * on first use and grown as needed).  Calls on one pool are serialised. */
aes_status aes_crypt_batched(aes_keypool* pool, const aes_msg* msgs, size_t nmsgs, const void* d_in,
                             void* d_out, size_t buf_bytes, void* cuda_stream);

/* One-shot form of aes_batch_run_iv (per-message IVs, Section II's V), through the same
 * internal batch context as aes_crypt_batched. */
aes_status aes_crypt_batched_iv(aes_keypool* pool, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs,
                                const void* d_in, void* d_out, size_t buf_bytes, void* cuda_stream);

/* The paper's CBC mode in its general form (Section II: key tensor K with a schedule per message,
 * IV matrix V with a row per message; App. A1/A4): many messages of different lengths, message i
 * under key-pool slot msgs[i].key_idx and IV ivs[16 i .. 16 i + 15] (host array of nmsgs x 16
 * bytes; NULL means zero IVs), chained over its blocks: C_j = Cipher_K(P_j xor C_{j-1}) with
 * C_{-1} = IV for msgs[i].dir = AES_ENCRYPT, P_j = InvCipher_K(C_j) xor C_{j-1} for AES_DECRYPT.
 * msgs and the buffers follow aes_batch_run's rules (offsets index both buffers, whole blocks,
 * AES-128/192/256 keys mixed).  Encryption is serial inside a message, so a long message is as
 * slow as its chain: up to 64 encrypted messages per SM run four lanes to a message, more run
 * one lane per message; decryption runs one lane per block.  A call with any
 * decryption message cannot run in place (AES_EINVAL).  Asynchronous on cuda_stream; the first
 * call on a pool allocates its descriptor buffers (kept with the pool, grown as needed).
 * Calls on one pool are serialised. */
aes_status aes_cbc_batched(aes_keypool* pool, const aes_msg* msgs, const uint8_t* ivs, size_t nmsgs, const void* d_in,
                           void* d_out, size_t buf_bytes, void* cuda_stream);

/* Batched encryption/decryption for callers that may not allocate device memory: for
 * example a plug-in whose host application owns all device memory and only lends it input
 * and output buffers, or a latency-critical path that cannot afford cudaMalloc's implicit
 * device-wide synchronisation.  The paper has no counterpart to this entry point.
 *
 * Same cipher and message rules as aes_batch_run, except that the caller passes the expanded
 * schedules directly (host array of nkeys <= 256 entries; msgs[i].key_idx indexes it) and at
 * most 4096 messages; larger counts are AES_EINVAL.  Nothing is allocated: all working data
 * (keys, descriptors, block starts, per-warp slices) lives in one static 416 KiB array in
 * device memory that the library declares, present on every device that loads the library
 * until the process exits.  The first call on a device may load the library's device code
 * (with lazy module loading that is where the array itself comes into being) and looks up
 * the array's device address; make that first call before any stream capture.  A call on a
 * stream that is being captured returns AES_EINVAL: the descriptors are staged in one shared
 * host buffer, so a captured copy would replay whatever that buffer held last.  The call may
 * block the host while it stages its descriptors from pageable memory; the device array is
 * updated in stream order.  All calls share the array: calls on one stream are ordered and
 * safe, calls that overlap on the GPU (other streams, no synchronisation) race on it and may
 * produce wrong output. */
aes_status aes_crypt_batched_noalloc(const aes_key_schedule* schedules, uint32_t nkeys, const aes_msg* msgs,
                                     size_t nmsgs, const void* d_in, void* d_out, size_t buf_bytes,
                                     void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Request server with continuous batching.  A host thread owned by the server admits queued
 * requests while device staging memory (the HBM budget) and in-flight slots are free, packs
 * them into one batched launch per CUDA stream, and starts the next batch on another stream
 * as soon as one is free, so requests that arrive while others run join the next launch
 * instead of waiting for a full drain.  Key schedules stay resident in the key pool.
 * ------------------------------------------------------------------------------------- */
typedef struct aes_server aes_server;

typedef struct {
  uint64_t hbm_budget;      /* device bytes for staging host payloads (>= 1 MiB) */
  uint32_t max_inflight;    /* requests admitted but not completed (>= 1) */
  uint32_t nstreams;        /* concurrent batches, 1..16 */
  uint32_t max_batch;       /* requests per launch, 1..65536 */
  uint32_t queue_capacity;  /* requests held at once, from submission until a poll reports them
                               finished (queued + running + finished-but-unpolled); beyond it
                               submit returns AES_EAGAIN (>= 1; rounded up to a power of two) */
  uint32_t fail_every;      /* fault injection for tests: every n-th launch fails on the host
                               without touching the GPU (its requests end FAILED); 0 = off */
  uint32_t linger_us;       /* microseconds the server's worker thread keeps polling (one host
                               core busy) after its last admission or completion before it
                               sleeps; requests that arrive within it skip a thread wake-up.
                               0 = sleep as soon as nothing is queued or running */
} aes_server_cfg;

typedef struct {
  uint32_t key_idx;        /* loaded key-pool slot */
  uint32_t dir;            /* AES_ENCRYPT or AES_DECRYPT */
  const void* src;         /* input: device pointer if src_on_device, else host pointer */
  void* dst;               /* output: device pointer if dst_on_device, else host pointer */
  uint64_t length;         /* bytes, a multiple of 16, > 0 */
  uint32_t src_on_device;  /* 1: src is device memory (16-byte aligned) */
  uint32_t dst_on_device;  /* 1: dst is device memory (16-byte aligned) */
} aes_request;

#define AES_REQ_PENDING 0
#define AES_REQ_DONE 1
#define AES_REQ_FAILED 2

typedef struct {
  uint64_t submitted, completed, failed, queued, inflight, launches;
  uint64_t bytes_completed;
  double p50_us, p99_us, max_us, mean_us; /* submit-to-completion latency of the completed requests
                                            (the most recent 2^22 since the last reset) */
  double gbps;                            /* bytes_completed / (last completion - first submit) */
  double mean_batch;                      /* requests per launch */
  double gbps_from_first_launch;          /* bytes_completed / (last completion - first launch) */
} aes_stats;

/* Starts a server on the current device over `pool` (which must outlive the server).  The
 * staging arena of cfg->hbm_budget bytes is allocated now; AES_ENOMEM if it does not fit. */
aes_status aes_server_create(const aes_server_cfg* cfg, aes_keypool* pool, aes_server** out);

/* Queues a copy of *req and returns its ticket.  The caller keeps src/dst alive and untouched
 * until the ticket is reported done.  AES_EAGAIN if queue_capacity requests are already held
 * (poll finished tickets to release them), AES_EINVAL for a bad request, AES_ENOMEM if it
 * needs more staging than the whole budget. */
aes_status aes_server_submit(aes_server* s, const aes_request* req, uint64_t* ticket);

/* Queues n requests at once (host array), all or none: AES_EAGAIN if fewer than n queue
 * places are free, AES_EINVAL / AES_ENOMEM if any request is bad (nothing is queued then).
 * tickets (host array of n) receives consecutive tickets in request order. */
aes_status aes_server_submit_many(aes_server* s, const aes_request* reqs, size_t n, uint64_t* tickets);

/* Waits up to timeout_us (0: do not wait; negative: no limit) for the ticket.  Returns AES_OK
 * with *state = AES_REQ_DONE or AES_REQ_FAILED (the ticket is then released),
 * AES_ETIMEDOUT with *state = AES_REQ_PENDING, or AES_ENOTFOUND for an unknown ticket. */
aes_status aes_server_poll(aes_server* s, uint64_t ticket, int64_t timeout_us, int* state);

/* Counters and latency percentiles since the last reset, written to *out (host). */
aes_status aes_server_stats(aes_server* s, aes_stats* out);
/* The same call under its earlier name. */
aes_status aes_server_stats_get(aes_server* s, aes_stats* out);
/* Clears the counters and the latency record. */
aes_status aes_server_stats_reset(aes_server* s);

/* Fails every queued request, waits for the batches on the GPU, joins the thread and frees
 * the server's memory.  NULL is a no-op. */
aes_status aes_server_destroy(aes_server* s);

#ifdef __cplusplus
}
#endif
#endif /* AESGB_H */
