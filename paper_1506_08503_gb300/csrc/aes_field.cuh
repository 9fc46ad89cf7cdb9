// aes_field.cuh -- GF(2^8) arithmetic and the AES tables derived from it at compile time.
//
// Everything here is constexpr and host+device: the S-box, its inverse and the T-tables
// are computed by the compiler from the field definition (arXiv:1506.08503 Section II:
// polynomial arithmetic modulo x^8 + x^4 + x^3 + x + 1), never typed in as literals.
//   - multiplication: Russian-peasant product with the xtime reduction (x * a);
//   - inverse: a^254 by square-and-multiply (the multiplicative group has order 255), with
//     0 -> 0 (App. A2);
//   - S-box: the affine map of App. A2 written with byte rotations, s = b ^ rotl(b,1) ^
//     rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ 0x63 (the circulant row 1 1 1 1 1 0 0 0 on
//     MSB-first vectors);
//   - inverse S-box: inv(rotl(x,1) ^ rotl(x,3) ^ rotl(x,6) ^ 0x05) (App. A5's circulant
//     row 0 1 0 1 0 0 1 0 and constant 0x05);
//   - T-tables: one S-box lookup fused with one column of the MixColumns matrix
//     circ(2 3 1 1) (App. A1), and with the InvMixColumns matrix circ(14 11 13 9) (App. A4).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define AES_HD __host__ __device__
#else
#define AES_HD
#endif

namespace aesgb {

AES_HD constexpr uint8_t gf_xtime(uint8_t a) {
  return static_cast<uint8_t>((a << 1) ^ ((a & 0x80u) ? 0x1Bu : 0u));
}

AES_HD constexpr uint8_t gf_mul(uint8_t a, uint8_t b) {
  uint8_t p = 0;
  for (int i = 0; i < 8; ++i) {
    if (b & 1u) p ^= a;
    a = gf_xtime(a);
    b >>= 1;
  }
  return p;
}

AES_HD constexpr uint8_t gf_pow(uint8_t a, int e) {
  uint8_t r = 1;
  while (e) {
    if (e & 1) r = gf_mul(r, a);
    a = gf_mul(a, a);
    e >>= 1;
  }
  return r;
}

AES_HD constexpr uint8_t gf_inv(uint8_t a) { return a ? gf_pow(a, 254) : 0; }

AES_HD constexpr uint8_t rotl8(uint8_t x, int s) {
  return static_cast<uint8_t>((x << s) | (x >> (8 - s)));
}

AES_HD constexpr uint8_t sbox(uint8_t x) {
  const uint8_t b = gf_inv(x);
  return static_cast<uint8_t>(b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63u);
}

AES_HD constexpr uint8_t inv_sbox(uint8_t x) {
  return gf_inv(static_cast<uint8_t>(rotl8(x, 1) ^ rotl8(x, 3) ^ rotl8(x, 6) ^ 0x05u));
}

AES_HD constexpr uint32_t pack4(uint8_t b0, uint8_t b1, uint8_t b2, uint8_t b3) {
  return uint32_t(b0) | (uint32_t(b1) << 8) | (uint32_t(b2) << 16) | (uint32_t(b3) << 24);
}

// A state column is a little-endian word: byte r is row r.
// Te0[x] = column 0 of circ(2 3 1 1) times S(x): rows (2s, s, s, 3s).
AES_HD constexpr uint32_t te0(uint8_t x) {
  const uint8_t s = sbox(x);
  return pack4(gf_mul(2, s), s, s, gf_mul(3, s));
}

// Td0[x] = column 0 of circ(14 11 13 9) times InvS(x): rows (14y, 9y, 13y, 11y).
AES_HD constexpr uint32_t td0(uint8_t x) {
  const uint8_t y = inv_sbox(x);
  return pack4(gf_mul(14, y), gf_mul(9, y), gf_mul(13, y), gf_mul(11, y));
}

struct FieldTables {
  uint32_t te0[256];   // encryption round table
  uint32_t td0[256];   // equivalent-inverse-cipher round table
  uint32_t s4[256];    // S(x) replicated in all four bytes (last encryption round)
  uint32_t is4[256];   // InvS(x) replicated in all four bytes (last decryption round)
  uint8_t s[256];
  uint8_t is[256];
};

AES_HD constexpr FieldTables make_field_tables() {
  FieldTables t{};
  for (int x = 0; x < 256; ++x) {
    const uint8_t s = sbox(static_cast<uint8_t>(x));
    const uint8_t y = inv_sbox(static_cast<uint8_t>(x));
    t.s[x] = s;
    t.is[x] = y;
    t.te0[x] = te0(static_cast<uint8_t>(x));
    t.td0[x] = td0(static_cast<uint8_t>(x));
    t.s4[x] = pack4(s, s, s, s);
    t.is4[x] = pack4(y, y, y, y);
  }
  return t;
}

// InvMixColumns of one column word (used to build the equivalent-inverse-cipher keys).
AES_HD constexpr uint32_t inv_mix_word(uint32_t w) {
  const uint8_t a0 = w & 0xFF, a1 = (w >> 8) & 0xFF, a2 = (w >> 16) & 0xFF, a3 = w >> 24;
  return pack4(gf_mul(14, a0) ^ gf_mul(11, a1) ^ gf_mul(13, a2) ^ gf_mul(9, a3),
               gf_mul(9, a0) ^ gf_mul(14, a1) ^ gf_mul(11, a2) ^ gf_mul(13, a3),
               gf_mul(13, a0) ^ gf_mul(9, a1) ^ gf_mul(14, a2) ^ gf_mul(11, a3),
               gf_mul(11, a0) ^ gf_mul(13, a1) ^ gf_mul(9, a2) ^ gf_mul(14, a3));
}

}  // namespace aesgb
