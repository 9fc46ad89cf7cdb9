// bitslice_host.cpp -- runs the bitsliced kernel's tile function (aes_bitslice.cuh: transposes,
// S-box networks, folded-key MixColumns, masks) as plain host C++, for the CPU test suite.
// Built by tests/test_bitslice_host.py with g++; not part of the library.
#include <cstdint>
#include <cstring>

#include "aes_bitslice.cuh"

namespace {

template <int NR, int DIR>
void run(const aesgb::bs::Masks& km, const uint8_t* in, uint8_t* out, size_t nblocks) {
  for (size_t t = 0; t < nblocks; t += 32) {
    uint32_t s[128];
    for (int j = 0; j < 32; ++j)
      for (int w = 0; w < 4; ++w) {
        uint32_t v = 0;
        if (t + j < nblocks) std::memcpy(&v, in + 16 * (t + j) + 4 * w, 4);  // little-endian words
        s[32 * w + j] = v;
      }
    aesgb::bs::crypt_tile<NR, DIR>(s, km.m[0]);
    for (int j = 0; j < 32 && t + j < nblocks; ++j)
      for (int w = 0; w < 4; ++w) std::memcpy(out + 16 * (t + j) + 4 * w, &s[32 * w + j], 4);
  }
}

}  // namespace

extern "C" int bs_host_crypt(const aes_key_schedule* ks, int dir, const uint8_t* iv, const uint8_t* in, uint8_t* out,
                             size_t nblocks) {
  static aesgb::bs::Masks km;
  aesgb::bs::fill_masks(km, *ks, dir, iv);
  const bool enc = dir == AES_ENCRYPT;
  switch (ks->nr) {
    case 10: enc ? run<10, AES_ENCRYPT>(km, in, out, nblocks) : run<10, AES_DECRYPT>(km, in, out, nblocks); return 0;
    case 12: enc ? run<12, AES_ENCRYPT>(km, in, out, nblocks) : run<12, AES_DECRYPT>(km, in, out, nblocks); return 0;
    case 14: enc ? run<14, AES_ENCRYPT>(km, in, out, nblocks) : run<14, AES_DECRYPT>(km, in, out, nblocks); return 0;
    default: return -1;
  }
}
