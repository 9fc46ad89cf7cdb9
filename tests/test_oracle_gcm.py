"""Pins for the oracle's Galois/Counter Mode (the counter-based mode that Section V of the paper
names as future work; defined by NIST SP 800-38D, not by the paper).

- The GF(2^128) product against polynomial arithmetic on Python integers (a carry-less
  product and long division by x^128 + x^7 + x^2 + x + 1, in the opposite bit order), and
  against the field laws: identity, commutativity, associativity, distributivity and
  a^(2^128 - 1) = 1.
- GHASH against its closed form, the polynomial sum X_1 H^n + ... + X_n H.
- Whole GCM encryption and decryption, bit-exact against OpenSSL's AES-GCM (through the
  `cryptography` package) for 128/192/256-bit keys, empty and ragged data and AAD.
- A flipped ciphertext block changes the tag by exactly delta * H^e.
- IVs other than 96 bits (J0 by GHASH of the IV): against OpenSSL for 8 to 128 bytes, and for
  lengths OpenSSL refuses (1, 7, 129 to 256 bytes) against GCM composed by definition from the
  separately pinned GHASH, counter mode and block cipher.
"""
import numpy as np
import pytest

POLY = (1 << 128) | 0x87  # x^128 + x^7 + x^2 + x + 1


def to_poly(block: np.ndarray) -> int:
    """Coefficient of x^i = bit i counted from the most significant bit of byte 0."""
    v = int.from_bytes(bytes(block), "big")
    return int(f"{v:0128b}"[::-1], 2)


def from_poly(p: int) -> np.ndarray:
    v = int(f"{p:0128b}"[::-1], 2)
    return np.frombuffer(v.to_bytes(16, "big"), dtype=np.uint8).copy()


def clmul_mod(a: int, b: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    for d in range(r.bit_length() - 1, 127, -1):
        if (r >> d) & 1:
            r ^= POLY << (d - 128)
    return r


def rnd(rng, n=16):
    return rng.integers(0, 256, n, dtype=np.uint8)


ONE = np.array([0x80] + [0] * 15, dtype=np.uint8)


def test_gf128_identity_and_reduction(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = rnd(rng)
        assert (orc.gf128_mul(a, ONE) == a).all() and (orc.gf128_mul(ONE, a) == a).all()
    x127 = np.zeros(16, dtype=np.uint8)
    x127[15] = 1
    x = np.zeros(16, dtype=np.uint8)
    x[0] = 0x40
    # x^127 * x = x^128 = 1 + x + x^2 + x^7: the bits 0..2 and 7 from the left, 0xE1 in byte 0
    want = np.zeros(16, dtype=np.uint8)
    want[0] = 0xE1
    assert (orc.gf128_mul(x127, x) == want).all()


def test_gf128_matches_polynomial_integers(orc):
    rng = np.random.default_rng(2)
    for _ in range(400):
        a, b = rnd(rng), rnd(rng)
        assert (orc.gf128_mul(a, b) == from_poly(clmul_mod(to_poly(a), to_poly(b)))).all()
    # sparse operands: single coefficients x^i * x^j
    for i in range(0, 128, 7):
        for j in range(0, 128, 11):
            assert (orc.gf128_mul(from_poly(1 << i), from_poly(1 << j)) == from_poly(clmul_mod(1 << i, 1 << j))).all()


def test_gf128_field_laws(orc):
    rng = np.random.default_rng(3)
    m = orc.gf128_mul
    for _ in range(100):
        a, b, c = rnd(rng), rnd(rng), rnd(rng)
        assert (m(a, b) == m(b, a)).all()
        assert (m(m(a, b), c) == m(a, m(b, c))).all()
        assert (m(a, b ^ c) == (m(a, b) ^ m(a, c))).all()


def test_gf128_fermat(orc):
    # the multiplicative group has order 2^128 - 1: a^(2^128 - 1) = 1 for every a != 0
    rng = np.random.default_rng(4)
    for _ in range(3):
        a = rnd(rng)
        acc, sq = ONE.copy(), a.copy()
        for _bit in range(128):  # 2^128 - 1 has all 128 low bits set
            acc = orc.gf128_mul(acc, sq)
            sq = orc.gf128_mul(sq, sq)
        assert (acc == ONE).all()


def power(orc, h, e):
    acc, sq = ONE.copy(), np.asarray(h, dtype=np.uint8).copy()
    while e:
        if e & 1:
            acc = orc.gf128_mul(acc, sq)
        sq = orc.gf128_mul(sq, sq)
        e >>= 1
    return acc


def test_ghash_closed_form(orc):
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 40):
        h = rnd(rng)
        x = rnd(rng, 16 * n)
        want = np.zeros(16, dtype=np.uint8)
        for i in range(n):
            want ^= orc.gf128_mul(x[16 * i:16 * i + 16], power(orc, h, n - i))
        assert (orc.ghash(h, x) == want).all()


def _aesgcm():
    return pytest.importorskip("cryptography.hazmat.primitives.ciphers.aead").AESGCM


@pytest.mark.parametrize("key_bytes", [16, 24, 32])
def test_gcm_matches_openssl(orc, key_bytes):
    AESGCM = _aesgcm()
    rng = np.random.default_rng(key_bytes)
    for length in (0, 1, 15, 16, 17, 100, 1000, 4099):
        for alen in (0, 5, 16, 33):
            key, iv = rnd(rng, key_bytes), rnd(rng, 12)
            pt, aad = rnd(rng, length), rnd(rng, alen)
            ct, tag = orc.gcm_crypt(key, iv, pt, aad)
            ref = AESGCM(key.tobytes()).encrypt(iv.tobytes(), pt.tobytes(), aad.tobytes() if alen else None)
            assert ct.tobytes() + tag.tobytes() == ref, (length, alen)
            back, tag2 = orc.gcm_crypt(key, iv, ct, aad, decrypt=True)
            assert (back == pt).all() and (tag2 == tag).all()
            # OpenSSL accepts the tag on decryption
            assert AESGCM(key.tobytes()).decrypt(iv.tobytes(), ref, aad.tobytes() if alen else None) == pt.tobytes()


def test_gcm_tag_difference_is_delta_times_power(orc):
    # the tag is linear in the ciphertext: flipping block j of c blocks (after a AAD blocks)
    # changes the tag by delta * H^(c - j + 1)
    rng = np.random.default_rng(6)
    key, iv = rnd(rng), rnd(rng, 12)
    c, aad = 50, rnd(rng, 40)
    ct = rnd(rng, 16 * c)
    h = orc.encrypt_blocks(key, np.zeros(16, dtype=np.uint8))
    _, t0 = orc.gcm_crypt(key, iv, ct, aad, decrypt=True)
    for j in (0, 17, c - 1):
        delta = rnd(rng)
        ct2 = ct.copy()
        ct2[16 * j:16 * j + 16] ^= delta
        _, t1 = orc.gcm_crypt(key, iv, ct2, aad, decrypt=True)
        assert ((t0 ^ t1) == orc.gf128_mul(delta, power(orc, h, c - j + 1))).all()


@pytest.mark.parametrize("iv_len", [8, 13, 16, 20, 32, 60, 64, 128])
def test_gcm_any_iv_length_matches_openssl(orc, iv_len):
    # IVs other than 96 bits take J0 = GHASH_H(IV, zero-padded, || 0^64 || bit length of IV)
    # (SP 800-38D); OpenSSL accepts 8 to 128 bytes
    AESGCM = _aesgcm()
    rng = np.random.default_rng(200 + iv_len)
    for key_bytes in (16, 24, 32):
        for length, alen in ((0, 0), (1, 0), (37, 5), (1000, 33)):
            key, iv = rnd(rng, key_bytes), rnd(rng, iv_len)
            pt, aad = rnd(rng, length), rnd(rng, alen)
            ct, tag = orc.gcm_crypt(key, iv, pt, aad)
            ref = AESGCM(key.tobytes()).encrypt(iv.tobytes(), pt.tobytes(), aad.tobytes() if alen else None)
            assert ct.tobytes() + tag.tobytes() == ref, (key_bytes, length, alen)
            back, tag2 = orc.gcm_crypt(key, iv, ct, aad, decrypt=True)
            assert (back == pt).all() and (tag2 == tag).all()


def _pad(b):
    return np.concatenate([b, np.zeros(-b.size % 16, dtype=np.uint8)])


def _lengths(a_bytes, c_bytes):
    return np.frombuffer(int(8 * a_bytes).to_bytes(8, "big") + int(8 * c_bytes).to_bytes(8, "big"), dtype=np.uint8)


@pytest.mark.parametrize("iv_len", [1, 7, 129, 200, 256])
def test_gcm_iv_outside_openssl_range_by_composition(orc, iv_len):
    # lengths OpenSSL refuses: GCM composed from the separately pinned GHASH, counter mode and
    # block cipher, following the definitions (J0 by GHASH; counters inc32(J0) + 1 + j, here
    # without a 32-bit wrap, which the test checks; tag = Cipher(J0) + GHASH(A, C, lengths))
    rng = np.random.default_rng(300 + iv_len)
    key, iv = rnd(rng, 16), rnd(rng, iv_len)
    pt, aad = rnd(rng, 100), rnd(rng, 20)
    h = orc.encrypt_blocks(key, np.zeros(16, dtype=np.uint8))
    j0 = orc.ghash(h, np.concatenate([_pad(iv), _lengths(0, iv_len)]))
    low = int.from_bytes(j0[12:].tobytes(), "big")
    assert low + 1 + 7 < 2 ** 32  # no inc32 wrap over the 7 data blocks
    ctr1 = j0.copy()
    ctr1[12:] = np.frombuffer((low + 1).to_bytes(4, "big"), dtype=np.uint8)
    stream = orc.ctr_crypt(key, ctr1, np.zeros(112, dtype=np.uint8))
    ct_ref = pt ^ stream[:100]
    tag_ref = orc.encrypt_blocks(key, j0) ^ orc.ghash(h, np.concatenate([_pad(aad), _pad(ct_ref), _lengths(20, 100)]))
    ct, tag = orc.gcm_crypt(key, iv, pt, aad)
    assert (ct == ct_ref).all() and (tag == tag_ref).all()
    # and the 96-bit special case really is special: a 12-byte IV does not take the GHASH route
    iv12 = rnd(rng, 12)
    j0_12 = np.concatenate([iv12, np.array([0, 0, 0, 1], dtype=np.uint8)])
    _, t12 = orc.gcm_crypt(key, iv12, b"", b"")
    assert (t12 == orc.encrypt_blocks(key, j0_12) ^ orc.ghash(h, _lengths(0, 0))).all()
