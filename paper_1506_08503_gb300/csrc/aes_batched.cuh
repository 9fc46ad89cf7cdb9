// aes_batched.cuh -- persistent T-table kernel over many messages, each with its own key.
//
// The paper keeps one key schedule per message (the tensor K, Section II) and processes all
// messages of a matrix together.  Here the messages of one direction are laid end to end in a
// virtual block space of G blocks (message m covers [start[m], start[m+1])), and that space
// is cut into one contiguous slice per warp.  The host places the cuts so that every warp has
// the same work in blocks x rounds (an AES-256 block costs 14 rounds, an AES-128 block 10),
// whatever the length and key-size mix, without atomics or per-tile searches.  Round keys sit
// in registers and are reloaded from the device key pool only when the key changes.  AES-128,
// -192 and -256 messages share a launch: the round count is read with the key.  Encryption
// and decryption share it too: the CTAs are split between them in proportion to their work.
#pragma once
#include "aes_ttable.cuh"

namespace aesgb {
namespace tt {

struct Cursor {
  uint32_t m = 0;
  uint64_t start = 0, end = 0, src = 0, dst = 0;
  uint32_t key = 0xFFFFFFFFu;
};

__device__ __forceinline__ uint64_t ldg64(const uint64_t* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}

// Message m with start[m] <= g < start[m + 1] (start strictly increasing, start[0] = 0).
__device__ __forceinline__ uint32_t find_msg(const uint64_t* start, uint32_t nmsgs, uint64_t g) {
  uint32_t lo = 0, hi = nmsgs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (ldg64(start + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" :: "l"(p));
}

__device__ __forceinline__ void open_msg(Cursor& c, const BatchDir& bd, uint32_t m) {
  c.m = m;
  c.start = ldg64(bd.start + m);
  c.end = ldg64(bd.start + m + 1);
  c.src = ldg64(&bd.msgs[m].src_block);
  c.dst = ldg64(&bd.msgs[m].dst_block);
  c.key = __ldg(&bd.msgs[m].key_idx);
}

// Moves the cursor forward until it holds block g (g below the direction's total).
__device__ __forceinline__ void seek(Cursor& c, const BatchDir& bd, uint64_t g) {
  while (g >= c.end) open_msg(c, bd, c.m + 1);
}

template <int DIR>
__device__ __forceinline__ void load_key(const PoolEntry* pool, uint32_t key, uint32_t (&kw)[kMaxRounds + 1][4],
                                         uint32_t (&kl)[4], int& nr) {
  const PoolEntry* e = pool + key;
  const uint4* kp = reinterpret_cast<const uint4*>(DIR == AES_ENCRYPT ? &e->enc[0][0] : &e->dec[0][0]);
#pragma unroll
  for (int r = 0; r < kMaxRounds; ++r) {
    const uint4 q = __ldg(kp + r);
    kw[r][0] = q.x; kw[r][1] = q.y; kw[r][2] = q.z; kw[r][3] = q.w;
  }
  nr = __ldg(&e->nr);
  const uint4 q = __ldg(kp + nr);
  kl[0] = q.x; kl[1] = q.y; kl[2] = q.z; kl[3] = q.w;
}

// Round keys in registers: NRF + 1 rows when every message of the direction has NRF rounds;
// for NRF = 0 (round counts mixed) the generic rows, the last key kl and the count nr read
// with the key.
template <int NRF>
struct KeyRegs {
  static constexpr int kRows = NRF ? NRF + 1 : kMaxRounds + 1;
  uint32_t kw[kRows][4];
  uint32_t kl[4];
  int nr;
};

template <int DIR, int NRF>
__device__ __forceinline__ void load_keys(const PoolEntry* pool, uint32_t key, KeyRegs<NRF>& k) {
  if constexpr (NRF == 0) {
    load_key<DIR>(pool, key, k.kw, k.kl, k.nr);
  } else {
    const PoolEntry* e = pool + key;
    const uint4* kp = reinterpret_cast<const uint4*>(DIR == AES_ENCRYPT ? &e->enc[0][0] : &e->dec[0][0]);
#pragma unroll
    for (int r = 0; r <= NRF; ++r) {
      const uint4 q = __ldg(kp + r);
      k.kw[r][0] = q.x; k.kw[r][1] = q.y; k.kw[r][2] = q.z; k.kw[r][3] = q.w;
    }
    k.nr = NRF;
  }
}

__device__ __forceinline__ uint4 ldg_iv(const uint4* p) { return __ldg(p); }

// XORs v into the round key that carries a message's IV: round key 0 for encryption
// (C = E(P ^ IV)), the last key for decryption (P = D(C) ^ IV; the equivalent inverse
// cipher's last key is K_0).  On a change of message within one key the old IV is taken out
// and the new one put in with one XOR of their difference.
template <int DIR, int NRF>
__device__ __forceinline__ void fold_iv(KeyRegs<NRF>& k, uint4 v) {
  uint32_t* w;
  if constexpr (DIR == AES_ENCRYPT) w = k.kw[0];
  else if constexpr (NRF == 0) w = k.kl;
  else w = k.kw[NRF];
  w[0] ^= v.x; w[1] ^= v.y; w[2] ^= v.z; w[3] ^= v.w;
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }

// Rounds 1..nr-1 of one block with the round keys in registers (nr = 10, 12 or 14; the
// branches are warp-uniform on the fast path).
template <int DIR>
__device__ __forceinline__ uint4 crypt_rt(uint4 v, const uint32_t (&kw)[kMaxRounds + 1][4], const uint32_t (&kl)[4],
                                          int nr, const char* sm, uint32_t lc) {
  uint32_t s0 = v.x ^ kw[0][0], s1 = v.y ^ kw[0][1], s2 = v.z ^ kw[0][2], s3 = v.w ^ kw[0][3];
#pragma unroll
  for (int r = 1; r < 10; ++r) tt_round<DIR>(s0, s1, s2, s3, kw[r][0], kw[r][1], kw[r][2], kw[r][3], sm, lc);
  if (nr > 10) {
#pragma unroll
    for (int r = 10; r < 12; ++r) tt_round<DIR>(s0, s1, s2, s3, kw[r][0], kw[r][1], kw[r][2], kw[r][3], sm, lc);
    if (nr > 12) {
#pragma unroll
      for (int r = 12; r < 14; ++r) tt_round<DIR>(s0, s1, s2, s3, kw[r][0], kw[r][1], kw[r][2], kw[r][3], sm, lc);
    }
  }
  return tt_final<DIR>(s0, s1, s2, s3, kl[0], kl[1], kl[2], kl[3], sm, lc);
}

template <int DIR, int NRF>
__device__ __forceinline__ uint4 crypt_keys(uint4 v, const KeyRegs<NRF>& k, const char* sm, uint32_t lc) {
  if constexpr (NRF == 0) {
    return crypt_rt<DIR>(v, k.kw, k.kl, k.nr, sm, lc);
  } else {
    uint32_t s0 = v.x ^ k.kw[0][0], s1 = v.y ^ k.kw[0][1], s2 = v.z ^ k.kw[0][2], s3 = v.w ^ k.kw[0][3];
#pragma unroll
    for (int r = 1; r < NRF; ++r) tt_round<DIR>(s0, s1, s2, s3, k.kw[r][0], k.kw[r][1], k.kw[r][2], k.kw[r][3], sm, lc);
    return tt_final<DIR>(s0, s1, s2, s3, k.kw[NRF][0], k.kw[NRF][1], k.kw[NRF][2], k.kw[NRF][3], sm, lc);
  }
}

// Warps step through their slice in windows of up to 32 * U blocks (lane l takes blocks
// base + l + 32u) that never cross a message boundary: a window ends where its message ends.
// The key, the round count and the source/destination bases are therefore the same for the
// whole warp (uniform registers and branches), and each lane enciphers U independent blocks.
// A window cut short by a message end leaves lanes idle; over lognormal lengths (median 4 KiB)
// that costs a few percent, less than per-lane keys at the boundaries would.  The next window
// of the same message is prefetched into L2 while the current one is enciphered, and during
// a message's last window the next message's key rows (L1) and first window (L2).  The host
// gives every warp the message holding its first block (warp_msg), so no warp searches.
// (Measured alternatives that were slower: the next window loaded into registers one window
// ahead; the first window issued before the table fill; a separate loop for whole windows,
// whose second copy of the unrolled rounds costs more in instruction fetch than it saves.)
// The work of CTA `cta` of the `ncta` CTAs given to one direction.
// NRF != 0: every message of the direction has NRF rounds (the host checks), so the round
// loop is fixed and the keys take NRF + 1 rows of registers.
// CHAIN (decryption only): the paper's CBC over whole messages, P_j = D(C_j) ^ C_{j-1} with
// C_{-1} = the message's IV (App. A4): each block's output is XORed with the previous input
// block of its message, or with bd.ivs[m] for the message's first block, instead of the IV
// riding on the keys.  The blocks are read through L1, so that the previous block, read by
// the neighbouring lane in the same window, is mostly an L1 hit.
template <int DIR, int THREADS, int U, int NRF = 0, bool CHAIN = false>
__device__ __forceinline__ void batched_body(uint64_t in_base, uint64_t out_base, const BatchDir& bd,
                                             const PoolEntry* pool, uint32_t cta, uint32_t ncta, uint32_t* smem) {
  static_assert(!CHAIN || DIR == AES_DECRYPT, "chaining is for decryption only");
  if (bd.total == 0) return;  // CTA-uniform, before any barrier
  fill_tables<DIR>(smem);
  __syncthreads();
  const char* sm = reinterpret_cast<const char*>(smem);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lc = lane * 4u;
  const uint64_t nwarps = uint64_t(ncta) * (THREADS / 32);
  const uint64_t w = (uint64_t(cta) * THREADS + threadIdx.x) >> 5;
  uint64_t gb, hi;
  if (bd.warp_gb) {
    gb = ldg64(bd.warp_gb + w);
    hi = ldg64(bd.warp_gb + w + 1);
  } else {
    hi = bd.total * (w + 1) / nwarps;
    gb = bd.total * w / nwarps;
  }
  if (gb >= hi) return;  // warp-uniform; no barrier follows

  KeyRegs<NRF> k;
  Cursor c;  // warp-uniform: the message holding block gb
  open_msg(c, bd, bd.warp_msg ? __ldg(bd.warp_msg + w) : find_msg(bd.start, bd.nmsgs, gb));
  load_keys<DIR, NRF>(pool, c.key, k);
  if (!CHAIN && bd.ivs) fold_iv<DIR, NRF>(k, ldg_iv(bd.ivs + c.m));
  constexpr uint32_t kWin = 32u * U;

  while (gb < hi) {
    if (gb >= c.end) {
      const uint32_t old = c.key, oldm = c.m;
      seek(c, bd, gb);
      if (c.key != old) {
        load_keys<DIR, NRF>(pool, c.key, k);
        if (!CHAIN && bd.ivs) fold_iv<DIR, NRF>(k, ldg_iv(bd.ivs + c.m));
      } else if (!CHAIN && bd.ivs) {
        fold_iv<DIR, NRF>(k, xor4(ldg_iv(bd.ivs + oldm), ldg_iv(bd.ivs + c.m)));
      }
    }
    uint64_t wend = gb + kWin;
    if (wend > hi) wend = hi;
    if (wend > c.end) wend = c.end;
    const uint4* src = reinterpret_cast<const uint4*>(in_base + (c.src + (gb - c.start)) * 16u);
    uint4* dst = reinterpret_cast<uint4*>(out_base + (c.dst + (gb - c.start)) * 16u);
    const uint32_t cnt = uint32_t(wend - gb);
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = u * 32u + lane;
      if constexpr (CHAIN) v[u] = i < cnt ? __ldg(src + i) : make_uint4(0u, 0u, 0u, 0u);
      else v[u] = i < cnt ? ld_block(src + i) : make_uint4(0u, 0u, 0u, 0u);
    }
    uint4 prev[CHAIN ? U : 1];
    if constexpr (CHAIN) {
      const bool first = gb == c.start;  // the window starts at the message's first block
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = u * 32u + lane;
        prev[u] = i >= cnt ? make_uint4(0u, 0u, 0u, 0u)
                  : (first && i == 0) ? ldg_iv(bd.ivs + c.m) : __ldg(src + i - 1);
      }
    }
    // the next window of the same message goes to L2 while this one is enciphered
    uint64_t nend = wend + kWin;
    if (nend > hi) nend = hi;
    if (nend > c.end) nend = c.end;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = kWin + u * 32u + lane;
      if (gb + i < nend) prefetch_l2(src + i);
    }
    if (wend == c.end && wend < hi) {
      // the message's last window, and the slice goes on into the next message: the next
      // key's rows go to L1 and the next message's first window to L2 while this window is
      // enciphered, so the switch does not wait on either (the next descriptor shares this
      // one's cache line three times in four)
      const BatchMsg* nm = bd.msgs + c.m + 1;
      const uint32_t nkey = __ldg(&nm->key_idx);
      const uint64_t nsrc = ldg64(&nm->src_block), nlen = ldg64(&nm->nblocks);
      const PoolEntry* e = pool + nkey;
      const char* kp = reinterpret_cast<const char*>(DIR == AES_ENCRYPT ? &e->enc[0][0] : &e->dec[0][0]);
      if (lane <= uint32_t(kMaxRounds)) prefetch_l1(kp + lane * 16u);
      const uint4* nsp = reinterpret_cast<const uint4*>(in_base + nsrc * 16u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = u * 32u + lane;
        if (i < nlen) prefetch_l2(nsp + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = crypt_keys<DIR, NRF>(v[u], k, sm, lc);
    if constexpr (CHAIN) {
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = xor4(v[u], prev[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = u * 32u + lane;
      if (i < cnt) st_block(dst + i, v[u]);
    }
    gb = wend;
  }
}

template <int DIR, int THREADS, int U>
__global__ void __launch_bounds__(THREADS, 1)
tt_batched_kernel(uint64_t in_base, uint64_t out_base, const BatchDir bd, const PoolEntry* pool) {
  extern __shared__ __align__(16) uint32_t smem[];
  batched_body<DIR, THREADS, U>(in_base, out_base, bd, pool, blockIdx.x, gridDim.x, smem);
}

// Both directions in one launch: CTAs [0, ge) encrypt, the others decrypt, so the two run
// side by side instead of one after the other (one tail, one launch).  Each CTA fills only
// its own direction's tables; the dynamic shared memory is sized for decryption.
// NRE / NRD: the round count of every encryption / decryption message, or 0 for mixed.
template <int THREADS, int U, int NRE = 0, int NRD = 0>
__global__ void __launch_bounds__(THREADS, 1)
tt_batched_dual(uint64_t in_base, uint64_t out_base, const BatchDir be, const BatchDir bdd, const PoolEntry* pool,
                uint32_t ge) {
  extern __shared__ __align__(16) uint32_t smem[];
  if (blockIdx.x < ge) batched_body<AES_ENCRYPT, THREADS, U, NRE>(in_base, out_base, be, pool, blockIdx.x, ge, smem);
  else batched_body<AES_DECRYPT, THREADS, U, NRD>(in_base, out_base, bdd, pool, blockIdx.x - ge, gridDim.x - ge, smem);
}

}  // namespace tt
}  // namespace aesgb
