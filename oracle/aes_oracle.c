/*
 * aes_oracle.c -- the slow, plain CPU oracle for AES as Kepner et al. build it from
 * Galois-field arithmetic (arXiv:1506.08503, Section II and Appendices A1-A5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  The product (the CUDA library) never calls,
 * links or includes anything here, and this file includes nothing of the product.
 *
 * Everything is computed from the field definition at initialisation time:
 *   - GF(2^8) addition is XOR and multiplication is the polynomial product reduced by
 *     x^8 + x^4 + x^3 + x + 1 (0x11B)                                     [Section II]
 *   - the multiplicative inverse is found by exhaustive search, with 0 -> 0  [App. A2]
 *   - the S-box is the affine map A*inv(x) + b, A = circulant(1 1 1 1 1 0 0 0),
 *     b = 0x63, on most-significant-bit-first bit vectors                     [App. A2]
 *   - the inverse S-box is inv(A'*x + b'), A' = circulant(0 1 0 1 0 0 1 0), b' = 0x05,
 *     with the one input whose affine image is 0 sent to 0                    [App. A5]
 *   - ShiftRows / InvShiftRows are the paper's byte gathers on the 16-byte
 *     column-major state                                          [Section II, App. A1, A4]
 *   - MixColumns / InvMixColumns multiply each 4-byte column by the circulant matrices
 *     circ(2 3 1 1) and circ(14 11 13 9) over GF(2^8)                  [App. A1, A4]
 *   - the AES-128 key schedule follows Appendix A3 (RotWord of the last column, SubBytes,
 *     round constant x^(r-1), running XOR over the four columns).  The 192- and 256-bit
 *     schedules are not in the paper (it treats 128-bit keys only, Section II); they follow
 *     the general Nk-word rule of the AES standard (FIPS-197 Section 5.2): every Nk-th word
 *     takes RotWord+SubWord+Rcon, and for Nk = 8 the word four after it takes SubWord.
 *   - encryption: add the IV, add round key 0, then Nr rounds of SubBytes, ShiftRows,
 *     MixColumns (skipped in the last round) and AddRoundKey                  [App. A1]
 *   - decryption: for r = Nr..1 add round key r, InvMixColumns unless r = Nr,
 *     InvShiftRows, InvSubBytes; then add round key 0 and the IV              [App. A4]
 *   - CBC chaining over the blocks of one message (the ciphertext of block j is the IV of
 *     block j+1)                                                     [Section II, App. A1, A4]
 *   - counter mode, which the paper leaves to future work (Section V): block i is
 *     P_i + Cipher(T + i), T the initial counter block read as a big-endian 128-bit integer
 *     (the usual counter increment of the AES modes); pinned against OpenSSL's CTR
 *   - the Galois/Counter Mode, the counter-based authenticated mode that Section V names as
 *     future work.  The paper does not define it; this follows NIST SP 800-38D: the
 *     GF(2^128) product bit by bit (its Algorithm 1), GHASH as Horner's rule (Algorithm 2),
 *     and GCM (Algorithms 4 and 5: J0 = IV || 0^31 || 1 for a 96-bit IV, else GHASH of
 *     the zero-padded IV and its bit length; data counters from inc32(J0); tag =
 *     Cipher(J0) + GHASH(A, C, lengths)); pinned against OpenSSL's GCM
 *
 * Parity is pinned by the test suite (GF brute force, field and S-box invariants, the
 * paper's worked examples, and bit-exact agreement with OpenSSL's AES).
 */
#include "aes_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* GF(2^8), Section II                                                                  */
/* ------------------------------------------------------------------------------------ */

#define AES_POLY 0x11Bu /* x^8 + x^4 + x^3 + x + 1, Section II */

uint8_t oracle_gf_add(uint8_t a, uint8_t b) { return (uint8_t)(a ^ b); }

/* Polynomial product of a and b with binary coefficients, then reduction modulo the AES
 * polynomial: the two steps of the worked example (x^7)(x^5) = x^12 -> x^7+x^5+x^3+x+1. */
uint8_t oracle_gf_mul(uint8_t a, uint8_t b) {
  uint32_t prod = 0;
  for (int i = 0; i < 8; ++i)
    if ((b >> i) & 1u) prod ^= (uint32_t)a << i; /* degree <= 14 */
  for (int d = 14; d >= 8; --d)
    if ((prod >> d) & 1u) prod ^= AES_POLY << (d - 8);
  return (uint8_t)prod;
}

/* Multiplicative inverse by exhaustive search; 0 has none and maps to 0 (App. A2 leaves
 * the entry for 0 untouched). */
uint8_t oracle_gf_inv(uint8_t a) {
  if (a == 0) return 0;
  for (int b = 1; b < 256; ++b)
    if (oracle_gf_mul(a, (uint8_t)b) == 1) return (uint8_t)b;
  return 0; /* unreachable: GF(2^8) is a field */
}

/* ------------------------------------------------------------------------------------ */
/* Affine maps over GF(2) on most-significant-bit-first vectors (App. A2, A5)            */
/* ------------------------------------------------------------------------------------ */

/* y = A x + b where A is the circulant matrix whose first row is `row` (each following
 * row is the previous one rotated right by one place) and x, y, b are 8-bit column
 * vectors whose first element is the most significant bit of the byte. */
static uint8_t affine_msb_first(const int row[8], const int b[8], uint8_t x) {
  int xv[8], yv[8];
  for (int i = 0; i < 8; ++i) xv[i] = (x >> (7 - i)) & 1;
  for (int i = 0; i < 8; ++i) {
    int acc = b[i];
    for (int j = 0; j < 8; ++j) {
      int aij = row[(j - i + 8) % 8]; /* circulant: A(i,j) = row((j - i) mod 8) */
      acc ^= aij & xv[j];
    }
    yv[i] = acc;
  }
  uint8_t y = 0;
  for (int i = 0; i < 8; ++i) y |= (uint8_t)(yv[i] << (7 - i));
  return y;
}

static const int SBOX_ROW[8] = {1, 1, 1, 1, 1, 0, 0, 0};    /* App. A2 */
static const int SBOX_B[8] = {0, 1, 1, 0, 0, 0, 1, 1};      /* App. A2: 0x63 */
static const int INVSBOX_ROW[8] = {0, 1, 0, 1, 0, 0, 1, 0}; /* App. A5 */
static const int INVSBOX_B[8] = {0, 0, 0, 0, 0, 1, 0, 1};   /* App. A5: 0x05 */

uint8_t oracle_affine(uint8_t x) { return affine_msb_first(SBOX_ROW, SBOX_B, x); }
uint8_t oracle_inv_affine(uint8_t x) { return affine_msb_first(INVSBOX_ROW, INVSBOX_B, x); }

/* ------------------------------------------------------------------------------------ */
/* Tables built once from the definitions                                                */
/* ------------------------------------------------------------------------------------ */

static uint8_t g_sbox[256], g_inv_sbox[256];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

static void build_tables(void) {
  for (int x = 0; x < 256; ++x) g_sbox[x] = oracle_affine(oracle_gf_inv((uint8_t)x)); /* A2 */
  /* A5: the inverse S-box is inv(A' x + b'), computed directly, not by inverting g_sbox */
  for (int x = 0; x < 256; ++x) g_inv_sbox[x] = oracle_gf_inv(oracle_inv_affine((uint8_t)x));
}

static void ensure_tables(void) { pthread_once(&g_once, build_tables); }

uint8_t oracle_sbox(uint8_t x) { ensure_tables(); return g_sbox[x]; }
uint8_t oracle_inv_sbox(uint8_t x) { ensure_tables(); return g_inv_sbox[x]; }

/* ------------------------------------------------------------------------------------ */
/* Round steps on the 16-byte state, byte i = row (i % 4), column (i / 4)                 */
/* ------------------------------------------------------------------------------------ */

/* ShiftRows as the paper's gather: state positions 2..16 (1-based) that move take their
 * value from the listed positions (App. A1, Section II "Shift rows"). */
static const int SR_DST[12] = {2, 3, 4, 6, 7, 8, 10, 11, 12, 14, 15, 16};
static const int SR_SRC[12] = {6, 11, 16, 10, 15, 4, 14, 3, 8, 2, 7, 12};
/* InvShiftRows, App. A4 */
static const int ISR_SRC[12] = {14, 11, 8, 2, 15, 12, 6, 3, 16, 10, 7, 4};

static void gather12(uint8_t s[16], const int src[12]) {
  uint8_t t[16];
  memcpy(t, s, 16);
  for (int k = 0; k < 12; ++k) s[SR_DST[k] - 1] = t[src[k] - 1];
}

void oracle_shift_rows(uint8_t s[16]) { gather12(s, SR_SRC); }
void oracle_inv_shift_rows(uint8_t s[16]) { gather12(s, ISR_SRC); }

void oracle_sub_bytes(uint8_t s[16]) {
  ensure_tables();
  for (int i = 0; i < 16; ++i) s[i] = g_sbox[s[i]];
}

void oracle_inv_sub_bytes(uint8_t s[16]) {
  ensure_tables();
  for (int i = 0; i < 16; ++i) s[i] = g_inv_sbox[s[i]];
}

/* Each column c (bytes 4c..4c+3) becomes M * column over GF(2^8), M the circulant matrix
 * with first row `row` (Section II "Multiply by M"; App. A1 row [2 3 1 1], App. A4 row
 * [14 11 13 9]). */
static void mix_with(uint8_t s[16], const uint8_t row[4]) {
  for (int c = 0; c < 4; ++c) {
    uint8_t col[4], out[4];
    memcpy(col, s + 4 * c, 4);
    for (int i = 0; i < 4; ++i) {
      uint8_t acc = 0;
      for (int j = 0; j < 4; ++j) acc = oracle_gf_add(acc, oracle_gf_mul(row[(j - i + 4) % 4], col[j]));
      out[i] = acc;
    }
    memcpy(s + 4 * c, out, 4);
  }
}

static const uint8_t MIX_ROW[4] = {2, 3, 1, 1};      /* App. A1 */
static const uint8_t INVMIX_ROW[4] = {14, 11, 13, 9}; /* App. A4 */

void oracle_mix_columns(uint8_t s[16]) { mix_with(s, MIX_ROW); }
void oracle_inv_mix_columns(uint8_t s[16]) { mix_with(s, INVMIX_ROW); }

void oracle_add(uint8_t s[16], const uint8_t k[16]) {
  for (int i = 0; i < 16; ++i) s[i] = oracle_gf_add(s[i], k[i]);
}

/* ------------------------------------------------------------------------------------ */
/* Key schedule (App. A3 for Nk = 4; FIPS-197 Section 5.2 rule for Nk = 6, 8)             */
/* ------------------------------------------------------------------------------------ */

/* Round constant x^(r-1) in GF(2^8) (App. A3), by repeated multiplication by x = 0x02. */
uint8_t oracle_rcon(int r) {
  uint8_t p = 1;
  for (int i = 1; i < r; ++i) p = oracle_gf_mul(p, 2);
  return p;
}

/* AES-128 schedule as Appendix A3 builds it, one 16-byte round key (four columns) at a
 * time: the new first column is SubBytes(RotWord(last column of the previous key)) plus
 * the round constant plus the previous first column, and every later column is the
 * previous key's column plus the new column before it. */
static void key_expand_128_rows(const uint8_t key[16], uint8_t rk[11][16]) {
  memcpy(rk[0], key, 16);
  for (int r = 1; r <= 10; ++r) {
    uint8_t t[4] = {rk[r - 1][13], rk[r - 1][14], rk[r - 1][15], rk[r - 1][12]};
    for (int j = 0; j < 4; ++j) t[j] = g_sbox[t[j]];
    t[0] = oracle_gf_add(t[0], oracle_rcon(r));
    for (int j = 0; j < 4; ++j) rk[r][j] = oracle_gf_add(rk[r - 1][j], t[j]);
    for (int c = 1; c < 4; ++c)
      for (int j = 0; j < 4; ++j) rk[r][4 * c + j] = oracle_gf_add(rk[r - 1][4 * c + j], rk[r][4 * (c - 1) + j]);
  }
}

/* General word rule of the AES standard (FIPS-197 Section 5.2) for Nk = 4, 6 or 8 key
 * words: w[i] = w[i-Nk] + t, where t = SubWord(RotWord(w[i-1])) + Rcon(i/Nk) when i is a
 * multiple of Nk, t = SubWord(w[i-1]) when Nk = 8 and i = 4 mod 8, else t = w[i-1]. */
int oracle_key_expand_words(const uint8_t* key, int nk, uint8_t* rk_out) {
  if (nk != 4 && nk != 6 && nk != 8) return -1;
  ensure_tables();
  const int nr = nk + 6;
  const int nwords = 4 * (nr + 1);
  uint8_t w[60][4];
  for (int i = 0; i < nk; ++i) memcpy(w[i], key + 4 * i, 4);
  for (int i = nk; i < nwords; ++i) {
    uint8_t t[4];
    memcpy(t, w[i - 1], 4);
    if (i % nk == 0) {
      uint8_t r0 = t[0];
      t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = r0;
      for (int j = 0; j < 4; ++j) t[j] = g_sbox[t[j]];
      t[0] = oracle_gf_add(t[0], oracle_rcon(i / nk));
    } else if (nk > 6 && i % nk == 4) {
      for (int j = 0; j < 4; ++j) t[j] = g_sbox[t[j]];
    }
    for (int j = 0; j < 4; ++j) w[i][j] = oracle_gf_add(w[i - nk][j], t[j]);
  }
  for (int i = 0; i < nwords; ++i) memcpy(rk_out + 4 * i, w[i], 4);
  return nr;
}

int oracle_key_expand(const uint8_t* key, int key_bits, uint8_t* rk_out) {
  ensure_tables();
  if (key_bits == 128) {
    uint8_t rk[11][16];
    key_expand_128_rows(key, rk);
    memcpy(rk_out, rk, sizeof(rk));
    return 10;
  }
  if (key_bits == 192) return oracle_key_expand_words(key, 6, rk_out);
  if (key_bits == 256) return oracle_key_expand_words(key, 8, rk_out);
  return -1;
}

/* ------------------------------------------------------------------------------------ */
/* Cipher and inverse cipher on one block (App. A1, A4)                                  */
/* ------------------------------------------------------------------------------------ */

void oracle_encrypt_block(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t in[16],
                          uint8_t out[16]) {
  uint8_t s[16];
  memcpy(s, in, 16);
  if (iv) oracle_add(s, iv);      /* add the IV */
  oracle_add(s, rk);              /* add round key 0 */
  for (int r = 1; r <= nr; ++r) {
    oracle_sub_bytes(s);
    oracle_shift_rows(s);
    if (r < nr) oracle_mix_columns(s); /* no MixColumns in the last round */
    oracle_add(s, rk + 16 * r);
  }
  memcpy(out, s, 16);
}

void oracle_decrypt_block(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t in[16],
                          uint8_t out[16]) {
  uint8_t s[16];
  memcpy(s, in, 16);
  for (int r = nr; r >= 1; --r) {
    oracle_add(s, rk + 16 * r);
    if (r < nr) oracle_inv_mix_columns(s);
    oracle_inv_shift_rows(s);
    oracle_inv_sub_bytes(s);
  }
  oracle_add(s, rk);           /* undo round 0 */
  if (iv) oracle_add(s, iv);   /* remove the IV */
  memcpy(out, s, 16);
}

/* ------------------------------------------------------------------------------------ */
/* Many independent blocks, split over threads (the paper's independent message groups,  */
/* Section IV)                                                                           */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  const uint8_t* rk;
  int nr;
  const uint8_t* iv;
  const uint8_t* in;
  uint8_t* out;
  size_t begin, end;
  int decrypt;
} slice_t;

static void* run_slice(void* p) {
  const slice_t* s = (const slice_t*)p;
  for (size_t i = s->begin; i < s->end; ++i) {
    if (s->decrypt) oracle_decrypt_block(s->rk, s->nr, s->iv, s->in + 16 * i, s->out + 16 * i);
    else oracle_encrypt_block(s->rk, s->nr, s->iv, s->in + 16 * i, s->out + 16 * i);
  }
  return NULL;
}

static int run_blocks(const uint8_t* rk, int nr, const uint8_t* iv, const uint8_t* in, uint8_t* out,
                      size_t nblocks, int nthreads, int decrypt) {
  ensure_tables();
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > nblocks) nthreads = nblocks ? (int)nblocks : 1;
  slice_t* sl = (slice_t*)calloc((size_t)nthreads, sizeof(slice_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!sl || !th) { free(sl); free(th); return -1; }
  for (int t = 0; t < nthreads; ++t) {
    sl[t].rk = rk; sl[t].nr = nr; sl[t].iv = iv; sl[t].in = in; sl[t].out = out;
    sl[t].begin = nblocks * (size_t)t / (size_t)nthreads;
    sl[t].end = nblocks * (size_t)(t + 1) / (size_t)nthreads;
    sl[t].decrypt = decrypt;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, run_slice, &sl[t]) != 0) break;
    started = t;
  }
  run_slice(&sl[0]);
  for (int t = started + 1; t < nthreads; ++t) run_slice(&sl[t]); /* any that failed to start */
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  free(sl); free(th);
  return 0;
}

int oracle_encrypt_blocks(const uint8_t* rk, int nr, const uint8_t* iv, const uint8_t* in,
                          uint8_t* out, size_t nblocks, int nthreads) {
  return run_blocks(rk, nr, iv, in, out, nblocks, nthreads, 0);
}

int oracle_decrypt_blocks(const uint8_t* rk, int nr, const uint8_t* iv, const uint8_t* in,
                          uint8_t* out, size_t nblocks, int nthreads) {
  return run_blocks(rk, nr, iv, in, out, nblocks, nthreads, 1);
}

/* CBC over one message of `nblocks` blocks (Section II: the ciphertext of a block is the IV
 * of the next; App. A1 encrypt, App. A4 decrypt). */
void oracle_cbc_encrypt(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t* in,
                        uint8_t* out, size_t nblocks) {
  uint8_t chain[16];
  memcpy(chain, iv, 16);
  for (size_t j = 0; j < nblocks; ++j) {
    oracle_encrypt_block(rk, nr, chain, in + 16 * j, out + 16 * j);
    memcpy(chain, out + 16 * j, 16);
  }
}

void oracle_cbc_decrypt(const uint8_t* rk, int nr, const uint8_t iv[16], const uint8_t* in,
                        uint8_t* out, size_t nblocks) {
  uint8_t chain[16], next[16];
  memcpy(chain, iv, 16);
  for (size_t j = 0; j < nblocks; ++j) {
    memcpy(next, in + 16 * j, 16); /* in == out is allowed */
    oracle_decrypt_block(rk, nr, chain, in + 16 * j, out + 16 * j);
    memcpy(chain, next, 16);
  }
}

/* Counter mode: out_i = in_i + Cipher(T + i), the counter block T a big-endian integer mod
 * 2^128 (Section V names counter-based modes as future work; the increment is the standard
 * one).  Encryption and decryption are the same operation. */
void oracle_ctr_crypt(const uint8_t* rk, int nr, const uint8_t ctr0[16], const uint8_t* in, uint8_t* out,
                      size_t nblocks) {
  uint8_t ctr[16], ks[16];
  memcpy(ctr, ctr0, 16);
  for (size_t j = 0; j < nblocks; ++j) {
    oracle_encrypt_block(rk, nr, NULL, ctr, ks);
    for (int b = 0; b < 16; ++b) out[16 * j + b] = oracle_gf_add(in[16 * j + b], ks[b]);
    for (int b = 15; b >= 0; --b) /* increment the 128-bit big-endian counter */
      if (++ctr[b] != 0) break;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Galois/Counter Mode (NIST SP 800-38D; Section V of the paper names it as future work)  */
/* ------------------------------------------------------------------------------------ */

/* Product in GF(2^128), one bit of x at a time (SP 800-38D Algorithm 1).  v runs through
 * y * x^i: multiplying by x moves every coefficient one bit towards the end of the block,
 * and a coefficient that leaves x^127 comes back as x^7 + x^2 + x + 1, which is 0xE1 in
 * byte 0. */
void oracle_gf128_mul(const uint8_t x[16], const uint8_t y[16], uint8_t z[16]) {
  uint8_t v[16], acc[16];
  memset(acc, 0, 16);
  memcpy(v, y, 16);
  for (int i = 0; i < 128; ++i) {
    if ((x[i / 8] >> (7 - i % 8)) & 1)
      for (int k = 0; k < 16; ++k) acc[k] ^= v[k];
    const int out = v[15] & 1;
    for (int k = 15; k > 0; --k) v[k] = (uint8_t)((v[k] >> 1) | (v[k - 1] << 7));
    v[0] >>= 1;
    if (out) v[0] ^= 0xE1;
  }
  memcpy(z, acc, 16);
}

/* GHASH (SP 800-38D Algorithm 2): Y_i = (Y_{i-1} + X_i) * H from Y_0 = 0. */
void oracle_ghash(const uint8_t h[16], const uint8_t* x, size_t nblocks, uint8_t y[16]) {
  uint8_t acc[16];
  memset(acc, 0, 16);
  for (size_t j = 0; j < nblocks; ++j) {
    for (int k = 0; k < 16; ++k) acc[k] ^= x[16 * j + k];
    oracle_gf128_mul(acc, h, acc);
  }
  memcpy(y, acc, 16);
}

/* One GHASH step over a block that may be short: the missing bytes count as zero. */
static void ghash_step(uint8_t acc[16], const uint8_t h[16], const uint8_t* blk, size_t nbytes) {
  for (size_t k = 0; k < nbytes; ++k) acc[k] ^= blk[k];
  oracle_gf128_mul(acc, h, acc);
}

/* GCM (SP 800-38D Algorithms 4 and 5).  H = Cipher(0^128).  J0 = IV || 0^31 || 1 for a
 * 96-bit IV; for any other length, J0 = GHASH_H(IV zero-padded to whole blocks || a block
 * holding 0^64 and the 64-bit bit length of the IV).  Data block j is XORed with
 * Cipher(J0 with its last 32 bits increased by 1 + j, mod 2^32); the hash runs over the AAD
 * and the ciphertext, each zero-padded to whole blocks, then the block [64-bit bit length of
 * AAD || 64-bit bit length of the ciphertext]; the tag is Cipher(J0) + that hash. */
void oracle_gcm_crypt_iv(const uint8_t* rk, int nr, const uint8_t* iv, size_t iv_len, const uint8_t* aad,
                         size_t aad_len, const uint8_t* in, uint8_t* out, size_t len, int decrypt, uint8_t tag[16]) {
  uint8_t h[16], j0[16], ctr[16], ks[16], acc[16], blk[16];
  memset(h, 0, 16);
  oracle_encrypt_block(rk, nr, NULL, h, h);
  if (iv_len == 12) {
    memcpy(j0, iv, 12);
    j0[12] = 0; j0[13] = 0; j0[14] = 0; j0[15] = 1;
  } else {
    memset(j0, 0, 16);
    for (size_t off = 0; off < iv_len; off += 16) ghash_step(j0, h, iv + off, iv_len - off < 16 ? iv_len - off : 16);
    const uint64_t ivbits = (uint64_t)iv_len * 8u;
    memset(blk, 0, 16);
    for (int k = 0; k < 8; ++k) blk[8 + k] = (uint8_t)(ivbits >> (56 - 8 * k));
    ghash_step(j0, h, blk, 16);
  }
  const uint32_t c0 = ((uint32_t)j0[12] << 24) | ((uint32_t)j0[13] << 16) | ((uint32_t)j0[14] << 8) | j0[15];
  memset(acc, 0, 16);
  for (size_t off = 0; off < aad_len; off += 16)
    ghash_step(acc, h, aad + off, aad_len - off < 16 ? aad_len - off : 16);
  memcpy(ctr, j0, 12);
  for (size_t j = 0; 16 * j < len; ++j) {
    const size_t off = 16 * j, nb = len - off < 16 ? len - off : 16;
    const uint32_t c = (uint32_t)(c0 + 1u + (uint32_t)j); /* inc32 wraps mod 2^32 */
    ctr[12] = (uint8_t)(c >> 24); ctr[13] = (uint8_t)(c >> 16); ctr[14] = (uint8_t)(c >> 8); ctr[15] = (uint8_t)c;
    oracle_encrypt_block(rk, nr, NULL, ctr, ks);
    memcpy(blk, in + off, nb); /* the ciphertext of a decryption, before in == out overwrites it */
    for (size_t k = 0; k < nb; ++k) out[off + k] = oracle_gf_add(in[off + k], ks[k]);
    ghash_step(acc, h, decrypt ? blk : out + off, nb);
  }
  const uint64_t abits = (uint64_t)aad_len * 8u, cbits = (uint64_t)len * 8u;
  for (int k = 0; k < 8; ++k) {
    blk[k] = (uint8_t)(abits >> (56 - 8 * k));
    blk[8 + k] = (uint8_t)(cbits >> (56 - 8 * k));
  }
  ghash_step(acc, h, blk, 16);
  oracle_encrypt_block(rk, nr, NULL, j0, ks);
  for (int k = 0; k < 16; ++k) tag[k] = (uint8_t)(ks[k] ^ acc[k]);
}

void oracle_gcm_crypt(const uint8_t* rk, int nr, const uint8_t iv[12], const uint8_t* aad, size_t aad_len,
                      const uint8_t* in, uint8_t* out, size_t len, int decrypt, uint8_t tag[16]) {
  oracle_gcm_crypt_iv(rk, nr, iv, 12, aad, aad_len, in, out, len, decrypt, tag);
}
