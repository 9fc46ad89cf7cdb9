/*
 * aes_oracle.h -- interface of the CPU oracle (test infrastructure only; see aes_oracle.c).
 * This header belongs to the oracle alone: the product library neither includes it nor
 * links the oracle, and the oracle includes nothing of the product.
 *
 * Conventions: a block is 16 bytes in the paper's column-major state order (byte i is row
 * i % 4, column i / 4).  A key schedule is (Nr + 1) round keys of 16 bytes, laid out
 * contiguously.  `iv` may be NULL (no IV added: plain ECB).
 */
#ifndef AES_ORACLE_H
#define AES_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* GF(2^8) with modulus x^8 + x^4 + x^3 + x + 1 (Section II) */
uint8_t oracle_gf_add(uint8_t a, uint8_t b);
uint8_t oracle_gf_mul(uint8_t a, uint8_t b);
uint8_t oracle_gf_inv(uint8_t a); /* exhaustive search, inv(0) = 0 (App. A2) */

/* affine maps of App. A2 (S-box) and App. A5 (inverse S-box) */
uint8_t oracle_affine(uint8_t x);
uint8_t oracle_inv_affine(uint8_t x);
uint8_t oracle_sbox(uint8_t x);     /* affine(inv(x)), App. A2 */
uint8_t oracle_inv_sbox(uint8_t x); /* inv(inv_affine(x)), App. A5 */

/* round steps on one 16-byte state, in place */
void oracle_sub_bytes(uint8_t s[16]);
void oracle_inv_sub_bytes(uint8_t s[16]);
void oracle_shift_rows(uint8_t s[16]);
void oracle_inv_shift_rows(uint8_t s[16]);
void oracle_mix_columns(uint8_t s[16]);
void oracle_inv_mix_columns(uint8_t s[16]);
void oracle_add(uint8_t s[16], const uint8_t k[16]);

/* key schedule: returns Nr (10, 12, 14) and writes 16*(Nr+1) bytes, or -1 on a bad size */
uint8_t oracle_rcon(int r); /* x^(r-1), App. A3 */
int oracle_key_expand(const uint8_t* key, int key_bits, uint8_t* rk_out);
int oracle_key_expand_words(const uint8_t* key, int nk, uint8_t* rk_out);

/* one block: C = Cipher(P + iv), P = InvCipher(C) + iv (App. A1 / A4 with one block) */
void oracle_encrypt_block(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t in[16],
                          uint8_t out[16]);
void oracle_decrypt_block(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t in[16],
                          uint8_t out[16]);

/* many independent blocks over `nthreads` host threads; in == out allowed; returns 0 */
int oracle_encrypt_blocks(const uint8_t* rk, int nr, const uint8_t* iv, const uint8_t* in,
                          uint8_t* out, size_t nblocks, int nthreads);
int oracle_decrypt_blocks(const uint8_t* rk, int nr, const uint8_t* iv, const uint8_t* in,
                          uint8_t* out, size_t nblocks, int nthreads);

/* CBC chaining over the nblocks blocks of ONE message (Section II, App. A1, A4) */
void oracle_cbc_encrypt(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t* in,
                        uint8_t* out, size_t nblocks);
void oracle_cbc_decrypt(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t* in,
                        uint8_t* out, size_t nblocks);

/* counter mode: out_i = in_i xor Cipher(ctr0 + i), ctr0 a big-endian 128-bit integer */
void oracle_ctr_crypt(const uint8_t* rk, int nr, const uint8_t ctr0[16], const uint8_t* in, uint8_t* out,
                      size_t nblocks);

/* GF(2^128) of the Galois/Counter Mode (NIST SP 800-38D): coefficient of x^i = bit i counted
 * from the most significant bit of byte 0, reduced by x^128 + x^7 + x^2 + x + 1 */
void oracle_gf128_mul(const uint8_t x[16], const uint8_t y[16], uint8_t z[16]);
/* GHASH_H over nblocks whole blocks: Y_0 = 0, Y_i = (Y_{i-1} + X_i) * H */
void oracle_ghash(const uint8_t h[16], const uint8_t* x, size_t nblocks, uint8_t y[16]);
/* AES-GCM with an IV of iv_len >= 1 bytes (96 bits: J0 = IV || 0^31 || 1; otherwise J0 by
 * GHASH of the IV and its length); decrypt != 0 hashes `in` (the ciphertext) instead of
 * `out`.  Writes len bytes to out and the 16-byte tag.  in == out is allowed. */
void oracle_gcm_crypt_iv(const uint8_t* rk, int nr, const uint8_t* iv, size_t iv_len, const uint8_t* aad,
                         size_t aad_len, const uint8_t* in, uint8_t* out, size_t len, int decrypt, uint8_t tag[16]);
/* the same with a 96-bit IV */
void oracle_gcm_crypt(const uint8_t* rk, int nr, const uint8_t iv[12], const uint8_t* aad, size_t aad_len,
                      const uint8_t* in, uint8_t* out, size_t len, int decrypt, uint8_t tag[16]);

#ifdef __cplusplus
}
#endif
#endif
