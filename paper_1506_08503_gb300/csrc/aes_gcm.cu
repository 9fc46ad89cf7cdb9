// aes_gcm.cu -- AES-GCM (Galois/Counter Mode, NIST SP 800-38D).
//
// Section V of the paper names counter-based authenticated modes (GCM) as future work.  GCM
// encrypts like counter mode -- data block j is XORed with the cipher of J0 (IV || 0^31 || 1
// for a 96-bit IV, else the GHASH of the padded IV and its length) whose last 32 bits are
// increased by 1 + j mod 2^32 -- and authenticates with GHASH, a
// polynomial in H = Cipher(0^128) over GF(2^128) modulo x^128 + x^7 + x^2 + x + 1:
//     S = X_1 H^m + X_2 H^(m-1) + ... + X_m H,    tag = Cipher(J0) + S,
// where X runs over the AAD and the ciphertext (each zero-padded to whole blocks) and a last
// block holding the two lengths in bits.  Coefficient of x^i = bit i of the block counted
// from the most significant bit of byte 0.
//
// GHASH is a serial Horner chain; here the sum is split instead.  With T threads (512 per
// CTA) and the n hashed blocks right-aligned in K*T positions (zeros in front), thread t
// takes positions t, t + T, t + 2T, ... and runs Horner's rule with the fixed multiplier
// Q = H^T, giving Y_t = sum_k X_(t+kT) Q^(K-1-k).  Then
//     sum_i X_i H^(n-i) = H * sum_t Y_t H^(T-1-t),
// and the last sum is a binary tree whose level j multiplies by H^(2^j): five levels between
// the lanes of a warp (shuffles), four between the 16 warps of a CTA, and between the CTAs
// as many as their count needs (none for one CTA, up to eight), in the CTA that finishes last.
//
// Multiplication by a fixed element M is linear, so it is one table lookup per 4-bit nibble
// of the other operand: Y * M = XOR over the 32 nibbles j of T_j[nibble_j(Y)], with
// T_j[v] = (v placed at nibble j) * M; a table is 32 x 16 entries of 16 bytes (8 KiB).  The
// tree's multipliers H^(2^j) use such tables, unreplicated.  The per-block multiplier Q is
// applied a byte at a time instead (Shoup's method): with B[b] = (b placed at byte 0) * Q,
// Y * Q = sum_k x^(8k) B[y_k], evaluated by Horner's rule from byte 15 down; multiplying by
// x^8 moves every byte up one place, and the byte pushed out of place 15 comes back as
// R[o] = o * x^128 reduced (a two-byte value, the same for every key).  That is 16 lookups of
// 16 bytes and 16 of 4 bytes per block, against 32 of 16 bytes with nibbles: 2.5 shared-memory
// wavefronts per block instead of 4, for a few more shifts.  B is replicated 8 times (lane l
// reads copy l mod 8, in its own four banks) and R 32 times (one copy per bank), so every
// lookup is conflict free whatever the data; the two take the 64 KiB beside the AES tables.
//
// One launch on the caller's stream.  Every CTA derives what it needs itself (H and
// Cipher(J0), H^(2^j) by repeated squaring, Q, the tables, from multiples M * x^i held in
// shared memory), runs the data pass (persistent, one CTA per SM: counter-mode AES with the
// T-table round code and a GHASH Horner step per block) and its tree; the CTA that finishes
// last, found with an atomic ticket (no CTA waits for another), combines the partial sums
// and writes the tag.  The caller's workspace holds only the partial sums and the ticket.
#include <cstring>

#include "aes_ttable.cuh"

namespace aesgb {
namespace {

using namespace tt;

// ---- workspace layout (bytes) ------------------------------------------------------------
constexpr int kMaxCtas = 256;
constexpr size_t kParts = 0;                        // one partial sum per CTA
constexpr size_t kCounter = kParts + kMaxCtas * 16;  // finished-CTA ticket (uint32)
constexpr size_t kWorkBytes = kCounter + 16;
constexpr int kThreads = 512;
constexpr uint32_t kAesSmem = 2 * kRegion;            // encryption T-tables (128 KiB)
constexpr uint32_t kMainSmem = kAesSmem + 65536;      // + the tables B and R of the Horner multiplier Q

// Element as four big-endian words, w0 the most significant (bytes 0..3): the view in which
// multiplying by x is a right shift.
struct Be {
  uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123u); }
__device__ __forceinline__ Be to_be(uint4 v) { return {bswap32(v.x), bswap32(v.y), bswap32(v.z), bswap32(v.w)}; }
__device__ __forceinline__ uint4 to_le(Be b) { return make_uint4(bswap32(b.w0), bswap32(b.w1), bswap32(b.w2), bswap32(b.w3)); }
__device__ __forceinline__ Be bxor(Be a, Be b) { return {a.w0 ^ b.w0, a.w1 ^ b.w1, a.w2 ^ b.w2, a.w3 ^ b.w3}; }
__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }

// b * x^r for 1 <= r <= 31: shift right by r; the r coefficients pushed past x^127 come back
// as O * (1 + x + x^2 + x^7), O being those bits at the top (x^0 ..) of the element.
__device__ __forceinline__ Be mulx_small(Be b, int r) {
  const uint32_t out = b.w3 << (32 - r);
  Be o{b.w0 >> r, __funnelshift_r(b.w1, b.w0, r), __funnelshift_r(b.w2, b.w1, r), __funnelshift_r(b.w3, b.w2, r)};
  uint64_t t = uint64_t(out) << 32;
  t ^= (t >> 1) ^ (t >> 2) ^ (t >> 7);
  o.w0 ^= uint32_t(t >> 32);
  o.w1 ^= uint32_t(t);
  return o;
}

__device__ Be mulx(Be b, int k) {  // b * x^k, 0 <= k < 128
  for (; k > 31; k -= 31) b = mulx_small(b, 31);
  return k ? mulx_small(b, k) : b;
}

// Bit u of a 32-bit word to bit 2u of a 64-bit word.
__device__ __forceinline__ uint64_t spread(uint32_t w) {
  uint64_t x = w;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

// a^2 = sum a_i x^(2i): the bits spread apart give x^0..x^127 (upper half) and x^128..x^255
// (lower half, B); then x^128 = 1 + x + x^2 + x^7 folds B back.
__device__ Be square(Be a) {
  const uint64_t r0 = spread(a.w0) << 1, r1 = spread(a.w1) << 1, r2 = spread(a.w2) << 1, r3 = spread(a.w3) << 1;
  const Be lo{uint32_t(r0 >> 32), uint32_t(r0), uint32_t(r1 >> 32), uint32_t(r1)};
  const Be b{uint32_t(r2 >> 32), uint32_t(r2), uint32_t(r3 >> 32), uint32_t(r3)};
  return bxor(bxor(lo, b), bxor(mulx_small(b, 1), bxor(mulx_small(b, 2), mulx_small(b, 7))));
}

// Entry v of nibble table j from the multiples mx[i] = M * x^i: the XOR of mx[4j + b] over
// the bits b of v, bit 3 of v standing for x^(4j).
__device__ __forceinline__ uint4 entry_from_multiples(const Be* mx, int j, int v) {
  Be acc{0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if ((v >> (3 - b)) & 1) acc = bxor(acc, mx[4 * j + b]);
  return to_le(acc);
}

// a * M for one warp (all 32 lanes, a warp-uniform) from the multiples mx[i] = M * x^i:
// lane l adds mx[i] for the set coefficients i = 4l .. 4l+3 of a, then the lanes XOR-reduce.
__device__ Be warp_mul(Be a, const Be* mx) {
  const int l = int(threadIdx.x & 31u);
  const uint32_t w = (l >> 3) == 0 ? a.w0 : (l >> 3) == 1 ? a.w1 : (l >> 3) == 2 ? a.w2 : a.w3;
  Be acc{0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int i = 4 * l + b;  // coefficient x^i: bit 31 - (i mod 32) of its word
    if ((w >> (31 - (i & 31))) & 1u) acc = bxor(acc, mx[i]);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    acc.w0 ^= __shfl_xor_sync(0xFFFFFFFFu, acc.w0, d);
    acc.w1 ^= __shfl_xor_sync(0xFFFFFFFFu, acc.w1, d);
    acc.w2 ^= __shfl_xor_sync(0xFFFFFFFFu, acc.w2, d);
    acc.w3 ^= __shfl_xor_sync(0xFFFFFFFFu, acc.w3, d);
  }
  return acc;
}

// y * M with M's unreplicated table (512 entries, entry j*16 + v).
__device__ __forceinline__ uint4 mul_tab(uint4 y, const uint4* tab) {
  uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const uint32_t w = j < 8 ? y.x : j < 16 ? y.y : j < 24 ? y.z : y.w;
    const uint32_t s = 8u * ((j >> 1) & 3) + ((j & 1) ? 0u : 4u);
    acc = xor4(acc, tab[j * 16 + ((w >> s) & 15u)]);
  }
  return acc;
}

// R[o]: the byte o pushed out of place 15 by a multiplication by x^8, reduced.  Bit 7 - m of o
// is the coefficient of x^(120 + m), which becomes x^(128 + m) = x^m (1 + x + x^2 + x^7); the
// result, of degree at most 14, is returned in the little-endian word view (bytes 0 and 1).
__device__ __forceinline__ uint32_t fold8(uint32_t o) {
  uint32_t r = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m)
    if ((o >> (7 - m)) & 1u) {
      const int e[4] = {m, m + 1, m + 2, m + 7};
#pragma unroll
      for (int q = 0; q < 4; ++q) r ^= 1u << (8 * (e[q] >> 3) + 7 - (e[q] & 7));
    }
  return r;
}

// y * Q a byte at a time (see the header): Z = B[y_15], then Z = Z x^8 + B[y_k] for k = 14
// down to 0, where Z x^8 is a left shift by 8 of the little-endian words plus R[byte 15].
// mb points at this lane's copy of B (entry b at b * 128), rb at its copy of R (entry o at
// o * 128); either offset is one shift and one AND of the byte.
__device__ __forceinline__ uint4 mul_q8(uint4 y, const char* mb, const char* rb) {
  const uint32_t w[4] = {y.x, y.y, y.z, y.w};
  auto boff = [&](int k) -> uint32_t {
    const int s = 8 * (k & 3);
    return (s >= 7 ? (w[k >> 2] >> (s - 7)) : (w[k >> 2] << (7 - s))) & 0x7F80u;
  };
  uint4 z = *reinterpret_cast<const uint4*>(mb + boff(15));
#pragma unroll
  for (int k = 14; k >= 0; --k) {
    const uint32_t r = *reinterpret_cast<const uint32_t*>(rb + ((z.w >> 17) & 0x7F80u));
    const uint4 m = *reinterpret_cast<const uint4*>(mb + boff(k));
    z.w = __funnelshift_l(z.z, z.w, 8) ^ m.w;
    z.z = __funnelshift_l(z.y, z.z, 8) ^ m.z;
    z.y = __funnelshift_l(z.x, z.y, 8) ^ m.y;
    z.x = (z.x << 8) ^ r ^ m.x;
  }
  return z;
}

__device__ __forceinline__ uint4 shfl_down4(uint4 v, int d) {
  return make_uint4(__shfl_down_sync(0xFFFFFFFFu, v.x, d), __shfl_down_sync(0xFFFFFFFFu, v.y, d),
                    __shfl_down_sync(0xFFFFFFFFu, v.z, d), __shfl_down_sync(0xFFFFFFFFu, v.w, d));
}

// Binary tree over the lanes of a warp, `levels` levels: level j pairs lane i (a multiple of
// 2^(j+1)) with lane i + 2^j as v_i * M_j + v_(i + 2^j), M_j the multiplier of table tabs[j].
// With M_j = M^(2^j), lane 0 ends with sum_l v_l M^(2^levels - 1 - l).
__device__ __forceinline__ uint4 lane_tree(uint4 v, const uint4* tabs, int levels) {
  const uint32_t lane = threadIdx.x & 31u;
  for (int j = 0; j < levels; ++j) {
    const uint4 o = shfl_down4(v, 1 << j);  // every lane takes part in the shuffle
    // only the lanes that keep a sum multiply: fewer lanes issue table loads at each level
    if ((lane & ((2u << j) - 1u)) == 0) v = xor4(mul_tab(v, tabs + j * 512), o);
  }
  return v;
}

// Up to 16 bytes from p (the rest zero); never reads past p[nb - 1].
__device__ __forceinline__ uint4 ld_partial(const uint8_t* p, uint32_t nb) {
  uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < 16; ++b)
    if (uint32_t(b) < nb) w[b >> 2] |= uint32_t(p[b]) << (8 * (b & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void st_partial(uint8_t* p, uint4 v, uint32_t nb) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int b = 0; b < 16; ++b)
    if (uint32_t(b) < nb) p[b] = uint8_t(w[b >> 2] >> (8 * (b & 3)));
}

__device__ __forceinline__ uint32_t byte_mask(uint32_t nb, int q) {  // bytes 4q.. of the first nb
  const int n = int(nb) - 4 * q;
  return n >= 4 ? 0xFFFFFFFFu : n <= 0 ? 0u : (1u << (8 * n)) - 1u;
}

struct GcmArgs {
  const uint4* in;
  uint4* out;
  const uint8_t* aad;
  uint64_t z;        // leading zero positions
  uint64_t a;        // AAD blocks
  uint64_t aad_len;  // bytes
  uint64_t len;      // data bytes
  uint32_t K;        // positions per thread
  uint4 j0;          // J0 of a 96-bit IV (IV || 0^31 || 1); ignored when IvHash::n > 0
  int decrypt;
  const uint8_t* expect;  // expected tag (decryption with verification), or nullptr
  int* ok;                // receives 1 if the computed tag equals *expect, else 0
};

// Writes the tag tg (little-endian words) to tag[0..15]; with an expected tag, also *ok = 1 if
// every byte matches, else 0 (all 16 bytes compared, no early exit).
__device__ void put_tag(uint4 tg, uint8_t* tag, const uint8_t* expect, int* ok) {
  const uint32_t tw[4] = {tg.x, tg.y, tg.z, tg.w};
  uint32_t diff = 0;
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const uint8_t v = uint8_t(tw[b >> 2] >> (8 * (b & 3)));
    tag[b] = v;
    if (expect) diff |= uint32_t(v ^ expect[b]);
  }
  if (expect) *ok = diff == 0u ? 1 : 0;
}

// For an IV other than 96 bits: the blocks GHASH runs over to give J0 (the IV zero-padded to
// whole blocks, then 0^64 and the IV's bit length), as little-endian words; n = 0 means that
// GcmArgs::j0 holds J0 directly.
constexpr int kMaxIvBytes = 256;
struct IvHash {
  uint4 b[kMaxIvBytes / 16 + 1];
  uint32_t n;
};

// J0 = GHASH_H over ivh's blocks, by the 32 lanes of one warp (all must call it): hmx (128
// entries of shared memory) receives the multiples H * x^i for warp_mul.
__device__ uint4 j0_from_iv(const IvHash& ivh, Be h, Be* hmx) {
  const int l = int(threadIdx.x & 31u);
  for (int i = l; i < 128; i += 32) hmx[i] = mulx(h, i);
  __syncwarp();
  Be y{0, 0, 0, 0};
  for (uint32_t b = 0; b < ivh.n; ++b) y = warp_mul(bxor(y, to_be(ivh.b[b])), hmx);
  return to_le(y);
}

// Counter block of data block j: J0 with its last 32 bits (big-endian) increased by 1 + j.
__device__ __forceinline__ uint4 counter_block(uint4 j0, uint64_t j) {
  return make_uint4(j0.x, j0.y, j0.z, bswap32(bswap32(j0.w) + 1u + uint32_t(j)));
}

// Builds, into tabs[k * 512 ..], the nibble tables of the multipliers ms[k] (k < count), using
// mx (count * 128 entries) as scratch for the multiples M * x^i.  All threads of the CTA
// call it; it ends with a barrier.
__device__ void build_tables(const Be* ms, int count, Be* mx, uint4* tabs) {
  for (uint32_t e = threadIdx.x; e < uint32_t(count) * 128u; e += blockDim.x) mx[e] = mulx(ms[e >> 7], int(e & 127u));
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < uint32_t(count) * 512u; e += blockDim.x)
    tabs[e] = entry_from_multiples(mx + (e >> 9) * 128, int((e >> 4) & 31u), int(e & 15u));
  __syncthreads();
}

// ---- the whole GCM in one launch ------------------------------------------------------------
// Every CTA: the AES T-tables; H = Cipher(0), Cipher(J0); the powers H^(2^j) by squaring;
// Q = H^T; Q's byte table B and the reduction table R (beside the T-tables); then the data
// pass (counter-mode AES
// and one GHASH Horner step per position); then the tree over its 512 threads.  The CTA that
// finishes last (an atomic ticket; nobody waits) combines the CTAs' partial sums and writes
// the tag.
template <int NR, int U>
__global__ void __launch_bounds__(kThreads, 1)
gcm_kernel(const GcmArgs g, const KeyWords kw, const IvHash ivh, char* work, uint8_t* tag, uint64_t abits,
           uint64_t cbits) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint4 s_he[2];  // Cipher(0) = H and Cipher(J0)
  __shared__ uint4 s_j0;
  __shared__ Be s_pow[18];
  __shared__ Be s_ms[9];
  __shared__ uint4 s_warp[kThreads / 32];
  __shared__ bool s_last;
  const uint32_t tid = threadIdx.x, lane = tid & 31u;
  char* smc = reinterpret_cast<char*>(smem);
  const char* sm = smc;
  const uint32_t lc = lane * 4u;
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  if (tid == 0) s_he[0] = crypt_block<NR, AES_ENCRYPT>(make_uint4(0, 0, 0, 0), kw, sm, lc);
  if (tid == 32 && ivh.n == 0) {
    s_j0 = g.j0;
    s_he[1] = crypt_block<NR, AES_ENCRYPT>(g.j0, kw, sm, lc);
  }
  __syncthreads();
  if (ivh.n) {  // uniform: J0 by GHASH of the IV, in the first warp (the Q region is free yet)
    if (tid < 32) {
      const uint4 j0 = j0_from_iv(ivh, to_be(s_he[0]), reinterpret_cast<Be*>(smc + kAesSmem));
      if (tid == 0) {
        s_j0 = j0;
        s_he[1] = crypt_block<NR, AES_ENCRYPT>(j0, kw, sm, lc);
      }
    }
    __syncthreads();
  }
  const uint4 j0 = s_j0;
  if (tid == 0) {
    // H^(2^j) for j <= 9 + LV, LV the last CTA's tree levels (2^LV >= gridDim.x): the in-CTA
    // tree takes j < 9, Q = H^T (T = 512 gridDim.x) its bits up to 9 + LV, the last tree 9 .. 8 + LV
    const int LV = gridDim.x > 1 ? 32 - __clz(gridDim.x - 1u) : 0;
    Be p = to_be(s_he[0]);
    s_pow[0] = p;
    for (int j = 1; j <= 9 + LV; ++j) s_pow[j] = p = square(p);
  }
  __syncthreads();
  // Q = H^T (T = gridDim.x * 512 < 2^18) from the multiples of the factors H^(2^b), kept in
  // the Q region until Q's own table is written there
  const uint32_t T = gridDim.x * kThreads;
  Be* qscratch = reinterpret_cast<Be*>(smc + kAesSmem);  // 18 x 128 multiples (36 KiB) at most
  for (uint32_t e = tid; e < 18u * 128u; e += kThreads)
    if ((T >> (e >> 7)) & 1u) qscratch[e] = mulx(s_pow[e >> 7], int(e & 127u));
  __syncthreads();
  if (tid < 32) {
    const int hi = 31 - __clz(T);
    Be q = s_pow[hi];
    for (int b = 0; b < hi; ++b)
      if ((T >> b) & 1u) q = warp_mul(q, qscratch + b * 128);
    if (tid == 0) s_ms[0] = q;
  }
  __syncthreads();
  Be* qmx = qscratch + 18 * 128;  // Q * x^i, i < 8, after the factors' (still inside the region)
  if (tid < 8) qmx[tid] = mulx(s_ms[0], int(tid));
  __syncthreads();
  // threads 0..255: entry tid of B (bit 7 - i of the byte is the coefficient of x^i);
  // threads 256..511: entry tid - 256 of R
  static_assert(kThreads == 512, "B and R take one entry per thread");
  uint4 be = make_uint4(0, 0, 0, 0);
  uint32_t re = 0;
  if (tid < 256) {
    Be acc{0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((tid >> (7 - i)) & 1u) acc = bxor(acc, qmx[i]);
    be = to_le(acc);
  } else {
    re = fold8(tid - 256u);
  }
  __syncthreads();  // every multiple is read before the tables overwrite the scratch
  if (tid < 256) {
    uint4* btab = reinterpret_cast<uint4*>(smc + kAesSmem);  // entry b, copy c at b * 128 + c * 16
#pragma unroll
    for (int c = 0; c < 8; ++c) btab[tid * 8 + c] = be;
  } else {
    uint4* rtab = reinterpret_cast<uint4*>(smc + kAesSmem + 32768);  // entry o, copy l at o * 128 + l * 4
#pragma unroll
    for (int c = 0; c < 8; ++c) rtab[(tid - 256u) * 8 + c] = make_uint4(re, re, re, re);
  }
  __syncthreads();
  const char* mb = sm + kAesSmem + (lane & 7u) * 16u;
  const char* rb = sm + kAesSmem + 32768 + lc;
  const uint64_t TT = T;
  const uint64_t t = uint64_t(blockIdx.x) * kThreads + tid;
  const uint64_t cblocks = (g.len + 15) / 16;

  uint4 y = make_uint4(0, 0, 0, 0);
  for (uint32_t k = 0; k < g.K; k += U) {
    uint4 x[U], ctr[U];
    int kind[U];  // 0 nothing, 1 AAD block, 2 data block
    uint64_t idx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t p = t + uint64_t(k + u) * TT;
      kind[u] = 0;
      idx[u] = 0;
      x[u] = make_uint4(0, 0, 0, 0);
      if (k + u < g.K && p >= g.z) {
        const uint64_t i = p - g.z;
        if (i < g.a) {
          kind[u] = 1;
          idx[u] = i;
          x[u] = 16 * (i + 1) <= g.aad_len ? ld_block(reinterpret_cast<const uint4*>(g.aad) + i)
                                           : ld_partial(g.aad + 16 * i, uint32_t(g.aad_len - 16 * i));
        } else if (i - g.a < cblocks) {
          const uint64_t jb = i - g.a;
          kind[u] = 2;
          idx[u] = jb;
          x[u] = 16 * (jb + 1) <= g.len ? ld_block(g.in + jb)
                                        : ld_partial(reinterpret_cast<const uint8_t*>(g.in) + 16 * jb, uint32_t(g.len - 16 * jb));
        }
      }
      ctr[u] = counter_block(j0, idx[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) ctr[u] = crypt_block<NR, AES_ENCRYPT>(ctr[u], kw, sm, lc);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uint4 h = x[u];
      if (kind[u] == 2) {
        const uint64_t jb = idx[u];
        const uint4 o = xor4(x[u], ctr[u]);
        if (16 * (jb + 1) <= g.len) {
          st_block(g.out + jb, o);
          if (!g.decrypt) h = o;
        } else {
          const uint32_t nb = uint32_t(g.len - 16 * jb);
          st_partial(reinterpret_cast<uint8_t*>(g.out) + 16 * jb, o, nb);
          if (!g.decrypt)
            h = make_uint4(o.x & byte_mask(nb, 0), o.y & byte_mask(nb, 1), o.z & byte_mask(nb, 2), o.w & byte_mask(nb, 3));
        }
      }
      if (k + u < g.K) y = xor4(mul_q8(y, mb, rb), h);
    }
  }

  // In-CTA tree: sum_i Y_i H^(511 - i) over the CTA's threads, with the tables of H^(2^j),
  // j = 0..8, built where the T-tables were (multiples as scratch in the Q region).
  __syncthreads();
  uint4* tabs = reinterpret_cast<uint4*>(smc);
  Be* mx = reinterpret_cast<Be*>(smc + kAesSmem);
  build_tables(s_pow, 9, mx, tabs);
  y = lane_tree(y, tabs, 5);
  if (lane == 0) s_warp[tid >> 5] = y;
  __syncthreads();
  if (tid < 32) {
    uint4 w = lane < kThreads / 32 ? s_warp[lane] : make_uint4(0, 0, 0, 0);
    w = lane_tree(w, tabs + 5 * 512, 4);
    if (lane == 0) {
      reinterpret_cast<uint4*>(work + kParts)[blockIdx.x] = w;
      __threadfence();  // the partial is visible device-wide before the ticket is taken
      const unsigned prev = atomicAdd(reinterpret_cast<unsigned*>(work + kCounter), 1u);
      s_last = prev == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!s_last) return;  // CTA-uniform; no barrier follows in the other CTAs
  __threadfence();

  // The last CTA: with LV levels (2^LV >= nb slots), CTA b's partial at slot 2^LV - nb + b
  // carries (H^512)^(2^LV - 1 - slot); a tree over the slots with the tables of H^(2^9) ..
  // H^(2^(8+LV)) (lanes of a warp for the first five levels, then the warps' sums), then the
  // tag.  A single CTA (LV = 0) needs no tree.
  const uint32_t nb = gridDim.x;
  const int LV = nb > 1 ? 32 - __clz(nb - 1u) : 0;
  const uint32_t S = 1u << LV;
  if (tid < uint32_t(LV)) s_ms[tid] = s_pow[9 + tid];
  if (tid == uint32_t(LV)) s_ms[LV] = s_pow[0];
  __syncthreads();
  build_tables(s_ms, LV + 1, mx, tabs);  // tabs[0..LV-1]: H^(2^9..2^(8+LV)), tabs[LV]: H
  const int l1 = LV < 5 ? LV : 5;
  const uint32_t lanes = S < 32u ? 32u : S;  // whole warps take part in the shuffles
  uint4 v = make_uint4(0, 0, 0, 0);
  if (tid < S && tid >= S - nb) v = __ldcg(reinterpret_cast<const uint4*>(work + kParts) + (tid - (S - nb)));
  if (tid < lanes) {
    v = lane_tree(v, tabs, l1);
    if (lane == 0) s_warp[tid >> 5] = v;
  }
  __syncthreads();
  if (tid < 32) {
    uint4 w = s_warp[0];
    if (LV > 5) {
      w = lane < (S >> 5) ? s_warp[lane] : make_uint4(0, 0, 0, 0);
      w = lane_tree(w, tabs + 5 * 512, LV - 5);
    }
    if (lane == 0) {
      const uint4* h_tab = tabs + LV * 512;
      const uint4 gsum = mul_tab(w, h_tab);  // sum_i X_i H^(n - i)
      const uint4 L = make_uint4(bswap32(uint32_t(abits >> 32)), bswap32(uint32_t(abits)), bswap32(uint32_t(cbits >> 32)),
                                 bswap32(uint32_t(cbits)));
      const uint4 S = mul_tab(xor4(gsum, L), h_tab);
      put_tag(xor4(s_he[1], S), tag, g.expect, g.ok);
      *reinterpret_cast<unsigned*>(work + kCounter) = 0u;  // ready for the next call on this workspace
    }
  }
}

// No hashed block at all (empty AAD and data): the tag is Cipher(J0) + (0 + L) * H with L = 0,
// i.e. Cipher(J0).  One warp (J0 by GHASH for an IV other than 96 bits), one thread writes.
template <int NR>
__global__ void __launch_bounds__(kThreads, 1) gcm_empty_kernel(const KeyWords kw, const uint4 j0_direct, const IvHash ivh,
                                                               uint8_t* tag, const uint8_t* expect, int* ok) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Be s_hmx[128];
  fill_tables<AES_ENCRYPT>(smem);
  __syncthreads();
  if (threadIdx.x < 32) {
    const char* sm = reinterpret_cast<const char*>(smem);
    const uint32_t lc = (threadIdx.x & 31u) * 4u;
    uint4 j0 = j0_direct;
    if (ivh.n) j0 = j0_from_iv(ivh, to_be(crypt_block<NR, AES_ENCRYPT>(make_uint4(0, 0, 0, 0), kw, sm, lc)), s_hmx);
    if (threadIdx.x == 0) put_tag(crypt_block<NR, AES_ENCRYPT>(j0, kw, sm, lc), tag, expect, ok);
  }
}

constexpr int kUnroll = 2;
using GcmFn = void (*)(const GcmArgs, const KeyWords, const IvHash, char*, uint8_t*, uint64_t, uint64_t);
using EmptyFn = void (*)(const KeyWords, const uint4, const IvHash, uint8_t*, const uint8_t*, int*);

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na && nb && x < y + nb && y < x + na;
}

}  // namespace
}  // namespace aesgb

using namespace aesgb;

extern "C" size_t aes_gcm_workspace_bytes(void) { return kWorkBytes; }

namespace {

aes_status gcm_launch(const aes_key_schedule* ks, const uint8_t* iv, size_t iv_len, const void* d_aad, size_t aad_len,
                      const void* d_in, void* d_out, size_t nbytes, int dir, uint8_t* d_tag, const uint8_t* d_expect,
                      int* d_ok, void* d_work, size_t work_bytes, void* cuda_stream) {
  if (!schedule_ok(ks)) return set_error(AES_EINVAL, "invalid key schedule (nr must be 10, 12 or 14)");
  if (dir != AES_ENCRYPT && dir != AES_DECRYPT) return set_error(AES_EINVAL, "dir must be AES_ENCRYPT or AES_DECRYPT");
  if (!iv || iv_len == 0 || iv_len > size_t(kMaxIvBytes))
    return set_error(AES_EINVAL, "GCM takes an IV of 1 to %d bytes", kMaxIvBytes);
  if (!d_tag) return set_error(AES_EINVAL, "null tag");
  if (!d_work || (reinterpret_cast<uintptr_t>(d_work) & 15u) || work_bytes < kWorkBytes)
    return set_error(AES_EINVAL, "workspace must be 16-byte aligned and at least %zu bytes", kWorkBytes);
  if (nbytes > (size_t(0xFFFFFFFFu) - 1u) * 16u)
    return set_error(AES_EINVAL, "GCM data is limited to 2^32 - 2 blocks");
  if (aad_len > (size_t(1) << 36)) return set_error(AES_EINVAL, "AAD is limited to 64 GiB");
  if (nbytes && (!d_in || !d_out)) return set_error(AES_EINVAL, "null buffer");
  if (aad_len && !d_aad) return set_error(AES_EINVAL, "null AAD");
  if (((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out) | reinterpret_cast<uintptr_t>(d_aad)) & 15u))
    return set_error(AES_EINVAL, "data and AAD buffers must be 16-byte aligned");
  if (d_in != d_out && overlaps(d_in, nbytes, d_out, nbytes))
    return set_error(AES_EINVAL, "input and output overlap without being identical");
  if (overlaps(d_out, nbytes, d_aad, aad_len)) return set_error(AES_EINVAL, "output overlaps the AAD");
  if (overlaps(d_work, kWorkBytes, d_in, nbytes) || overlaps(d_work, kWorkBytes, d_out, nbytes) ||
      overlaps(d_work, kWorkBytes, d_aad, aad_len) || overlaps(d_work, kWorkBytes, d_tag, 16))
    return set_error(AES_EINVAL, "workspace overlaps a buffer");
  if (d_expect && (overlaps(d_expect, 16, d_out, nbytes) || overlaps(d_expect, 16, d_tag, 16) ||
                   overlaps(d_expect, 16, d_work, kWorkBytes) || overlaps(d_ok, sizeof(int), d_out, nbytes) ||
                   overlaps(d_ok, sizeof(int), d_tag, 16) || overlaps(d_ok, sizeof(int), d_work, kWorkBytes) ||
                   overlaps(d_ok, sizeof(int), d_expect, 16)))
    return set_error(AES_EINVAL, "expected tag or ok flag overlaps a buffer the call writes");
  const DeviceInfo* di = current_device_info();
  if (!di) return AES_ECUDA;
  if (di->smem_optin < int(kMainSmem)) return set_error(AES_EINVAL, "device has too little shared memory for GCM");

  const uint64_t a = (aad_len + 15) / 16, c = (nbytes + 15) / 16, n = a + c;
  const int max_ctas = di->sms < kMaxCtas ? di->sms : kMaxCtas;
  const uint64_t want = (n + kThreads - 1) / kThreads;  // at least one position per thread
  const uint32_t nb = n == 0 ? 0u : uint32_t(want < 1 ? 1 : want > uint64_t(max_ctas) ? uint64_t(max_ctas) : want);
  const uint32_t T = (nb ? nb : 1u) * kThreads;
  // J0 directly for a 96-bit IV; otherwise the blocks its GHASH runs over (in the kernel)
  uint4 j0{0u, 0u, 0u, 0u};
  IvHash ivh{};
  if (iv_len == 12) {
    uint32_t ivw[3];
    std::memcpy(ivw, iv, 12);
    j0 = make_uint4(ivw[0], ivw[1], ivw[2], 0x01000000u);  // bytes 12..15 = 0, 0, 0, 1
  } else {
    const size_t nblk = (iv_len + 15) / 16;
    uint8_t bytes[(kMaxIvBytes / 16 + 1) * 16] = {};
    std::memcpy(bytes, iv, iv_len);
    const uint64_t ivbits = uint64_t(iv_len) * 8u;
    for (int k = 0; k < 8; ++k) bytes[nblk * 16 + 8 + k] = uint8_t(ivbits >> (56 - 8 * k));
    for (size_t i = 0; i <= nblk; ++i) {
      uint32_t w[4];
      for (int q = 0; q < 4; ++q)
        w[q] = uint32_t(bytes[16 * i + 4 * q]) | (uint32_t(bytes[16 * i + 4 * q + 1]) << 8) |
               (uint32_t(bytes[16 * i + 4 * q + 2]) << 16) | (uint32_t(bytes[16 * i + 4 * q + 3]) << 24);
      ivh.b[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    ivh.n = uint32_t(nblk + 1);
  }
  const KeyWords kw = enc_key_words(*ks, nullptr);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  char* work = static_cast<char*>(d_work);

  cudaError_t e;
  if (nb == 0) {  // nothing hashed: the tag is Cipher(J0)
    EmptyFn k0 = ks->nr == 10 ? gcm_empty_kernel<10> : ks->nr == 12 ? gcm_empty_kernel<12> : gcm_empty_kernel<14>;
    aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(k0), kAesSmem);
    if (ast != AES_OK) return ast;
    k0<<<1, kThreads, kAesSmem, st>>>(kw, j0, ivh, d_tag, d_expect, d_ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "GCM launch");
    return AES_OK;
  }
  GcmFn k = ks->nr == 10 ? gcm_kernel<10, kUnroll> : ks->nr == 12 ? gcm_kernel<12, kUnroll> : gcm_kernel<14, kUnroll>;
  {
    aes_status ast = ensure_kernel_smem(reinterpret_cast<const void*>(k), kMainSmem);
    if (ast != AES_OK) return ast;
  }
  // the finished-CTA ticket starts at zero (the last CTA also puts it back)
  if ((e = cudaMemsetAsync(work + kCounter, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(GCM ticket)");
  GcmArgs g;
  g.in = static_cast<const uint4*>(d_in);
  g.out = static_cast<uint4*>(d_out);
  g.aad = static_cast<const uint8_t*>(d_aad);
  g.K = uint32_t((n + T - 1) / T);
  g.z = uint64_t(g.K) * T - n;
  g.a = a;
  g.aad_len = aad_len;
  g.len = nbytes;
  g.j0 = j0;
  g.decrypt = dir == AES_DECRYPT;
  g.expect = d_expect;
  g.ok = d_ok;
  k<<<nb, kThreads, kMainSmem, st>>>(g, kw, ivh, work, d_tag, uint64_t(aad_len) * 8u, uint64_t(nbytes) * 8u);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "GCM launch");
  return AES_OK;
}

}  // namespace

extern "C" aes_status aes_gcm_crypt(const aes_key_schedule* ks, const uint8_t* iv, size_t iv_len, const void* d_aad,
                                    size_t aad_len, const void* d_in, void* d_out, size_t nbytes, int dir, uint8_t* d_tag,
                                    void* d_work, size_t work_bytes, void* cuda_stream) {
  clear_error();
  return gcm_launch(ks, iv, iv_len, d_aad, aad_len, d_in, d_out, nbytes, dir, d_tag, nullptr, nullptr, d_work, work_bytes,
                    cuda_stream);
}

extern "C" aes_status aes_gcm_decrypt_verify(const aes_key_schedule* ks, const uint8_t* iv, size_t iv_len,
                                             const void* d_aad, size_t aad_len, const void* d_in, void* d_out,
                                             size_t nbytes, const uint8_t* d_expected_tag, int* d_ok, uint8_t* d_tag,
                                             void* d_work, size_t work_bytes, void* cuda_stream) {
  clear_error();
  if (!d_expected_tag || !d_ok) return set_error(AES_EINVAL, "null expected tag or ok flag");
  if (reinterpret_cast<uintptr_t>(d_ok) & (alignof(int) - 1)) return set_error(AES_EINVAL, "ok flag must be int-aligned");
  return gcm_launch(ks, iv, iv_len, d_aad, aad_len, d_in, d_out, nbytes, AES_DECRYPT, d_tag, d_expected_tag, d_ok, d_work,
                    work_bytes, cuda_stream);
}
