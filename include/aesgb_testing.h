/* aesgb_testing.h -- test hooks into host-side logic of libaesgb.so.  They touch no GPU, so the
 * CPU test suite can check the logic directly.  Not part of the stable interface: signatures
 * may change with the implementation they expose. */
#ifndef AESGB_TESTING_H
#define AESGB_TESTING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The batched launch's per-warp slicing of one direction: n messages of nblocks[i] blocks and
 * rounds[i] rounds (10, 12 or 14) laid end to end, cut into nw slices of equal work in
 * blocks x rounds.  Writes the first block of every slice to gb[0..nw] (gb[nw] = total) and
 * the message holding it to msg[0..nw-1].  Returns 0, or -1 for bad arguments (n = 0, a
 * message without blocks, rounds outside 10/12/14, n > 2^20). */
int aes_testing_weighted_slices(const uint64_t* nblocks, const int8_t* rounds, size_t n, uint64_t nw, uint64_t* gb,
                                uint32_t* msg);

/* The request server's staging allocator (first fit over [0, size), 256-byte granules, freed
 * neighbours coalesced), driven by nops operations: ops[i] > 0 allocates ops[i] bytes and
 * writes the offset (or -1 when nothing fits) to results[i]; ops[i] = -(j + 1) frees the
 * allocation made by operation j (nothing, if it failed; results[i] = 0).  Returns 0, or -1
 * for a bad operation (0, a free of no earlier allocation, a second free). */
int aes_testing_arena(size_t size, const int64_t* ops, size_t nops, int64_t* results);

/* The single-key launch tuner's JSON cache: stores (impl, threads, unroll, us) under `sig` in
 * the file at `path` (keeping other entries), or looks `sig` up.  lookup returns 1 when found
 * (a compiled candidate), 0 otherwise; store returns 0. */
int aes_testing_tune_cache_store(const char* path, const char* sig, int impl, int threads, int unroll, double us);
int aes_testing_tune_cache_lookup(const char* path, const char* sig, int* impl, int* threads, int* unroll);

/* The launch shape of CBC encryption with four lanes per chain for `chains` chains on a device
 * of `sms` SMs: CTA threads, the warps of a CTA that run chains, grid, and chains per warp.
 * Returns 0, or -1 for chains = 0 or sms < 1. */
int aes_testing_cols_shape(uint64_t chains, int sms, unsigned* threads, unsigned* wpc, unsigned* grid, unsigned* cpw);

#ifdef __cplusplus
}
#endif
#endif
