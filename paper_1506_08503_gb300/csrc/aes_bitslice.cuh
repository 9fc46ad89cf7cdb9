// aes_bitslice.cuh -- the bitsliced (gate-level, constant-time) AES rounds on 32 blocks at a
// time, shared by the CUDA kernel (aes_bitslice.cu) and, compiled as plain host C++, by the
// CPU test that runs the same code on the host against the oracle.
//
// The paper computes SubBytes as GF(2^8) inversion plus an affine map and MixColumns as a
// GF(2^8) matrix product (Section II, App. A1-A5).  Here both are Boolean circuits evaluated
// on "planes": a thread owns 32 blocks, and its 128 registers s[8b + i] hold bit i of state
// byte b for all 32 blocks (bit j of a plane = block j).  Then
//   * SubBytes is the tower-field S-box network of three-input tables (aes_bitslice_sbox.cuh,
//     77 LOP3 instructions) on 8 planes, 16 times;
//   * ShiftRows is a renaming of registers (no instruction);
//   * MixColumns is a network of three-input XORs with the next round key folded in (see
//     mix_column), and InvMixColumns is MixColumns o P (see inv_mix_shift);
//   * AddRoundKey of the first and last round XORs each plane with an all-zeros or all-ones
//     mask held in the constant bank (kernel parameter); the other rounds' keys ride inside
//     MixColumns, so they cost no instruction.
// No table, no data-dependent branch or address: time is independent of data and key.
#pragma once
#include <cstdint>
#include <cstring>

#include "aes_bitslice_sbox.cuh"
#include "aes_field.cuh"
#include "aesgb.h"

#if defined(__CUDACC__)
#define BS_FN __host__ __device__ __forceinline__
#else
#define BS_FN inline
#endif

namespace aesgb {
namespace bs {

constexpr int kBsMaxRounds = 14;

// prmt/__byte_perm in its default mode: byte i of the result is byte (s >> 4i) & 7 of y:x.
BS_FN uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __byte_perm(x, y, s);
#else
  const uint64_t v = (uint64_t(y) << 32) | x;
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= uint32_t((v >> (8 * ((s >> (4 * i)) & 7u))) & 0xFFu) << (8 * i);
  return r;
#endif
}

struct Masks {
  uint32_t m[kBsMaxRounds + 1][128];
};

// (a & M) | (b & ~M) for a constant mask M.  On the device one LOP3 with M as its immediate:
// written in C, the compiler moved the mask across the transposes' shifts and spent two
// instructions per output.
template <uint32_t M>
BS_FN uint32_t select_bits(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "n"(M));
  return d;
#else
  return (a & M) | (b & ~M);
#endif
}

// One shift stage of the transpose: swaps the J-bit sub-blocks between rows k and k + J.
template <int J>
BS_FN void swap_stage(uint32_t* a) {
  constexpr uint32_t m = J == 4 ? 0x0F0F0F0Fu : J == 2 ? 0x33333333u : 0x55555555u;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k & J) continue;
    const uint32_t x = a[k], y = a[k + J];
    a[k] = select_bits<m>(x, y << J);
    a[k + J] = select_bits<m>(x >> J, y);
  }
}

// 32x32 bit transpose in place: afterwards bit j of a[p] is the old bit p of a[j].
BS_FN void transpose32(uint32_t* a) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t x = a[k], y = a[k + 16];
    a[k] = byte_perm(x, y, 0x5410u);
    a[k + 16] = byte_perm(x, y, 0x7632u);
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k & 8) continue;
    const uint32_t x = a[k], y = a[k + 8];
    a[k] = byte_perm(x, y, 0x6240u);
    a[k + 8] = byte_perm(x, y, 0x7351u);
  }
  swap_stage<4>(a);
  swap_stage<2>(a);
  swap_stage<1>(a);
}

BS_FN uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }

BS_FN void ark(uint32_t* s, const uint32_t* k) {
#pragma unroll
  for (int i = 0; i < 128; ++i) s[i] ^= k[i];
}

BS_FN void sub_bytes(uint32_t* s) {
#pragma unroll
  for (int b = 0; b < 16; ++b) sbox_planes(s[8 * b], s[8 * b + 1], s[8 * b + 2], s[8 * b + 3], s[8 * b + 4], s[8 * b + 5], s[8 * b + 6], s[8 * b + 7]);
}

BS_FN void inv_sub_bytes(uint32_t* s) {
#pragma unroll
  for (int b = 0; b < 16; ++b) inv_sbox_planes(s[8 * b], s[8 * b + 1], s[8 * b + 2], s[8 * b + 3], s[8 * b + 4], s[8 * b + 5], s[8 * b + 6], s[8 * b + 7]);
}

// byte (r, c) of the state is byte r + 4c; ShiftRows reads row r of column c + r
BS_FN constexpr int sr_src(int r, int c) { return r + 4 * ((c + r) & 3); }
BS_FN constexpr int isr_src(int r, int c) { return r + 4 * ((c - r) & 3); }

// MixColumns of one column with a round key folded in (App. A1's circulant circ(2 3 1 1)):
//   out_r = 2 a_r + 3 a_r+1 + a_r+2 + a_r+3 + k_r = x t_r + a_r+1 + t_r+2,  t_r = a_r + a_r+1 + c_r,
// where the constants c (one byte per row, cm = 8 mask planes per row) satisfy
// x c_r + c_r+2 = k_r, so the key costs no instruction: c_r enters the three-input XOR that
// forms t_r.  xtime on planes moves plane 7 into planes 0, 1, 3, 4 (x^8 = x^4 + x^3 + x + 1),
// so out_r bit i is a three-input XOR for i = 0, 2, 5, 6, 7 and two for i = 1, 3, 4:
// 19 instructions per row.
BS_FN void mix_column(const uint32_t* const (&a)[4], const uint32_t* cm, uint32_t* const (&o)[4]) {
  uint32_t c[32];  // the column's folding constants, read as eight 16-byte vectors on the device
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint4 v = reinterpret_cast<const uint4*>(cm)[q];
    c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
  }
#else
  for (int i = 0; i < 32; ++i) c[i] = cm[i];
#endif
  uint32_t t[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) t[r][i] = xor3(a[r][i], a[(r + 1) & 3][i], c[8 * r + i]);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint32_t* u = t[r];
    const uint32_t* b = a[(r + 1) & 3];
    const uint32_t* v = t[(r + 2) & 3];
    o[r][0] = xor3(u[7], b[0], v[0]);
    o[r][1] = xor3(u[0], u[7], b[1]) ^ v[1];
    o[r][2] = xor3(u[1], b[2], v[2]);
    o[r][3] = xor3(u[2], u[7], b[3]) ^ v[3];
    o[r][4] = xor3(u[3], u[7], b[4]) ^ v[4];
    o[r][5] = xor3(u[4], b[5], v[5]);
    o[r][6] = xor3(u[5], b[6], v[6]);
    o[r][7] = xor3(u[6], b[7], v[7]);
  }
}

// Encryption rounds 1..Nr-1 after SubBytes: ShiftRows (a renaming), then MixColumns with the
// next round key folded in (cm: 128 mask words, row r of column c at 8 (r + 4c)), into n.
BS_FN void shift_mix(const uint32_t* s, uint32_t* n, const uint32_t* cm) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t* const a[4] = {s + 8 * sr_src(0, c), s + 8 * sr_src(1, c), s + 8 * sr_src(2, c), s + 8 * sr_src(3, c)};
    uint32_t* const o[4] = {n + 8 * (4 * c), n + 8 * (4 * c + 1), n + 8 * (4 * c + 2), n + 8 * (4 * c + 3)};
    mix_column(a, cm + 32 * c, o);
  }
}

// The last encryption round: ShiftRows and AddRoundKey.
BS_FN void shift_ark(const uint32_t* s, uint32_t* n, const uint32_t* k) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = s[8 * sr_src(r, c) + i] ^ k[8 * (r + 4 * c) + i];
}

// InvMixColumns with a key folded in, then InvShiftRows, into n.  circ(14 11 13 9) equals
// circ(2 3 1 1) * circ(5 0 4 0) over GF(2^8), so InvMixColumns = MixColumns o P with
// P(col)_r = a_r + x^2 (a_r + a_r+2): the pair (a_h, a_h+2) shares u = a_h + a_h+2 and w = x^2 u,
// whose bits are u6, u6+u7, u0+u7, u1+u6, u2+u6+u7, u3+u7, u4, u5 (bits 0..7).
// InvMixColumns(s + K) = MixColumns(P(s)) + InvMixColumns(K): cm holds the constants for
// the key InvMixColumns(K_r), folded as in mix_column.
BS_FN void inv_mix_shift(const uint32_t* s, uint32_t* n, const uint32_t* cm) {
  uint32_t m[128];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t* a[4] = {s + 8 * (4 * c), s + 8 * (4 * c + 1), s + 8 * (4 * c + 2), s + 8 * (4 * c + 3)};
    uint32_t b[4][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t* x = a[h];
      const uint32_t* y = a[h + 2];
      uint32_t u[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) u[i] = x[i] ^ y[i];
      const uint32_t w4 = xor3(u[2], u[6], u[7]);
      b[h][0] = x[0] ^ u[6];
      b[h][1] = xor3(x[1], u[6], u[7]);
      b[h][2] = xor3(x[2], u[0], u[7]);
      b[h][3] = xor3(x[3], u[1], u[6]);
      b[h][4] = x[4] ^ w4;
      b[h][5] = xor3(x[5], u[3], u[7]);
      b[h][6] = xor3(x[6], x[4], y[4]);
      b[h][7] = xor3(x[7], x[5], y[5]);
      b[h + 2][0] = y[0] ^ u[6];
      b[h + 2][1] = xor3(y[1], u[6], u[7]);
      b[h + 2][2] = xor3(y[2], u[0], u[7]);
      b[h + 2][3] = xor3(y[3], u[1], u[6]);
      b[h + 2][4] = y[4] ^ w4;
      b[h + 2][5] = xor3(y[5], u[3], u[7]);
      b[h + 2][6] = xor3(y[6], x[4], y[4]);
      b[h + 2][7] = xor3(y[7], x[5], y[5]);
    }
    const uint32_t* const bb[4] = {b[0], b[1], b[2], b[3]};
    uint32_t* const o[4] = {m + 8 * (4 * c), m + 8 * (4 * c + 1), m + 8 * (4 * c + 2), m + 8 * (4 * c + 3)};
    mix_column(bb, cm + 32 * c, o);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = m[8 * isr_src(r, c) + i];
}

BS_FN void inv_shift(const uint32_t* s, uint32_t* n) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) n[8 * (r + 4 * c) + i] = s[8 * isr_src(r, c) + i];
}

// Masks row r (km + 128 r): round 0 = K_0 (+ IV), rows 1..Nr-1 = the folding constants of
// K_r, row Nr = K_Nr.  The middle rounds run as a loop, not unrolled: sixteen S-box networks
// and a MixColumns are some 1,600 instructions per round, and the whole cipher unrolled
// (25,000 for AES-128) would not stay in the instruction caches (8 warps per SM streaming
// through it stalled on instruction fetch more than on anything else).
template <int NR>
BS_FN void encrypt_planes(uint32_t* s, const uint32_t* km) {
  ark(s, km);
#pragma unroll 1
  for (int r = 1; r < NR; ++r) {
    sub_bytes(s);
    uint32_t n[128];
    shift_mix(s, n, km + 128 * r);
#pragma unroll
    for (int i = 0; i < 128; ++i) s[i] = n[i];
  }
  sub_bytes(s);
  uint32_t n[128];
  shift_ark(s, n, km + 128 * NR);
#pragma unroll
  for (int i = 0; i < 128; ++i) s[i] = n[i];
}

// The paper's inverse cipher order (App. A4): for r = Nr..1 add K_r, InvMixColumns unless
// r = Nr, InvShiftRows, InvSubBytes; then add K_0 (which carries the IV).  For r < Nr the key
// addition rides inside InvMixColumns (masks row r = the folding constants of
// InvMixColumns(K_r)).  The middle rounds run as a loop, as in encrypt_planes.
template <int NR>
BS_FN void decrypt_planes(uint32_t* s, const uint32_t* km) {
  ark(s, km + 128 * NR);
  {
    uint32_t n[128];
    inv_shift(s, n);
#pragma unroll
    for (int i = 0; i < 128; ++i) s[i] = n[i];
  }
  inv_sub_bytes(s);
#pragma unroll 1
  for (int r = NR - 1; r >= 1; --r) {
    uint32_t n[128];
    inv_mix_shift(s, n, km + 128 * r);
#pragma unroll
    for (int i = 0; i < 128; ++i) s[i] = n[i];
    inv_sub_bytes(s);
  }
  ark(s, km);
}

// One tile: words[32 w + j] is word w (bytes 4w..4w+3) of block j, in and out.  Four 32x32
// transposes turn the 32 blocks into 128 planes and back around the rounds.
template <int NR, int DIR>
BS_FN void crypt_tile(uint32_t* s, const uint32_t* km) {
#pragma unroll
  for (int q = 0; q < 4; ++q) transpose32(s + 32 * q);
  if constexpr (DIR == AES_ENCRYPT) encrypt_planes<NR>(s, km);
  else decrypt_planes<NR>(s, km);
#pragma unroll
  for (int q = 0; q < 4; ++q) transpose32(s + 32 * q);
}

// 128 mask words from 16 bytes: word 8b + i is all ones when bit i of byte b is set.
inline void expand_masks(uint32_t* m, const uint8_t* bytes) {
  for (int b = 0; b < 16; ++b)
    for (int i = 0; i < 8; ++i) m[8 * b + i] = ((bytes[b] >> i) & 1u) ? 0xFFFFFFFFu : 0u;
}

// The constants c_0..c_3 of one column with x c_r + c_r+2 = k_r (rows mod 4), so that adding
// c_r inside MixColumns' t_r adds k_r to its output: pairing rows r and r + 2,
// c_r = (k_r+2 + x k_r) / (1 + x^2) and c_r+2 = k_r + x c_r.
inline void fold_column(const uint8_t* k, uint8_t* c) {
  constexpr uint8_t inv5 = gf_inv(0x05);  // 1 + x^2
  for (int r = 0; r < 2; ++r) {
    c[r] = gf_mul(static_cast<uint8_t>(k[r + 2] ^ gf_xtime(k[r])), inv5);
    c[r + 2] = static_cast<uint8_t>(k[r] ^ gf_xtime(c[r]));
  }
}

inline void fill_masks(Masks& km, const aes_key_schedule& ks, int dir, const uint8_t* iv) {
  const int nr = ks.nr;
  uint8_t k0[16];
  for (int b = 0; b < 16; ++b) k0[b] = static_cast<uint8_t>(ks.rk[0][b] ^ (iv ? iv[b] : 0));  // IV rides on K0
  expand_masks(km.m[0], k0);
  expand_masks(km.m[nr], ks.rk[nr]);
  for (int r = 1; r < nr; ++r) {
    uint8_t k[16], c[16];
    std::memcpy(k, ks.rk[r], 16);
    if (dir == AES_DECRYPT)
      for (int col = 0; col < 4; ++col) {
        uint32_t w = 0;
        for (int j = 0; j < 4; ++j) w |= uint32_t(k[4 * col + j]) << (8 * j);
        w = inv_mix_word(w);
        for (int j = 0; j < 4; ++j) k[4 * col + j] = static_cast<uint8_t>(w >> (8 * j));
      }
    for (int col = 0; col < 4; ++col) fold_column(k + 4 * col, c + 4 * col);
    expand_masks(km.m[r], c);
  }
}

}  // namespace bs
}  // namespace aesgb
