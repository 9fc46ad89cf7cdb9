"""GPU parity for AES-GCM (the counter-based authenticated mode that Section V of the paper
names as future work; NIST SP 800-38D) against the oracle's GCM, with 96-bit IVs and with IVs
of other lengths (J0 by GHASH of the IV, in the kernel).

Output bytes and tags are compared exactly.  Sizes span one to many CTAs, several positions
per thread, ragged final blocks of data and AAD, and the empty cases.  At 1 GiB the
ciphertext is checked on sampled blocks against the oracle's cipher of the counter blocks,
decryption must return the plaintext and the same tag, and the tag of a sparse ciphertext is
compared with its closed form sum_j C_j H^(c - j + 1) + L H + Cipher(J0), evaluated with the
oracle's GF(2^128) product.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [(0, 0), (0, 13), (1, 0), (16, 16), (15, 17), (4095, 33), (16 * 2048 + 5, 100),
         (16 * 77_824 + 9, 0), (16 * (3 * 77_824 + 1000) + 3, 4100)]


@pytest.mark.parametrize("key_bits", [128, 192, 256])
@pytest.mark.parametrize("nbytes,aad_len", CASES)
def test_gcm_matches_oracle(aes, orc, cuda, key_bits, nbytes, aad_len):
    if key_bits != 128 and nbytes > 16 * 100_000:
        pytest.skip("large sizes run with AES-128 only")
    rng = np.random.default_rng(nbytes * 7 + aad_len + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    iv = rng.integers(0, 256, 12, dtype=np.uint8)
    pt = rng.integers(0, 256, nbytes, dtype=np.uint8)
    aad = rng.integers(0, 256, aad_len, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    want_ct, want_tag = orc.gcm_crypt(key, iv, pt, aad)
    ct, tag = aes.gcm(dev(pt), ks, iv.tobytes(), aad=dev(aad) if aad_len else None)
    assert (host(ct) == want_ct).all()
    assert (host(tag) == want_tag).all()
    back, tag2 = aes.gcm(ct, ks, iv.tobytes(), aad=dev(aad) if aad_len else None, dir="decrypt")
    assert (host(back) == pt).all() and (host(tag2) == want_tag).all()


@pytest.mark.parametrize("iv_len", [1, 8, 11, 13, 16, 17, 64, 128, 255, 256])
@pytest.mark.parametrize("nbytes,aad_len", [(0, 0), (0, 20), (37, 5), (16 * 300_000 + 3, 33)])
def test_gcm_any_iv_length(aes, orc, cuda, iv_len, nbytes, aad_len):
    rng = np.random.default_rng(1000 * iv_len + nbytes % 997 + aad_len)
    key_bits = (128, 192, 256)[iv_len % 3]
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    iv = rng.integers(0, 256, iv_len, dtype=np.uint8)
    pt = rng.integers(0, 256, nbytes, dtype=np.uint8)
    aad = rng.integers(0, 256, aad_len, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    want_ct, want_tag = orc.gcm_crypt(key, iv, pt, aad)
    ct, tag = aes.gcm(dev(pt), ks, iv.tobytes(), aad=dev(aad) if aad_len else None)
    assert (host(ct) == want_ct).all()
    assert (host(tag) == want_tag).all()
    back, tag2 = aes.gcm(ct, ks, iv.tobytes(), aad=dev(aad) if aad_len else None, dir="decrypt")
    assert (host(back) == pt).all() and (host(tag2) == want_tag).all()


@pytest.mark.parametrize("iv_len,nbytes,aad_len", [(12, 16 * 50_000 + 5, 21), (12, 0, 0), (20, 100, 0), (7, 0, 9)])
def test_gcm_open_checks_the_tag_on_the_device(aes, orc, cuda, iv_len, nbytes, aad_len):
    rng = np.random.default_rng(77 + iv_len + nbytes)
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    iv = rng.integers(0, 256, iv_len, dtype=np.uint8).tobytes()
    pt = rng.integers(0, 256, nbytes, dtype=np.uint8)
    aad = rng.integers(0, 256, aad_len, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes())
    ct, tag = orc.gcm_crypt(key, iv, pt, aad)
    d_aad = dev(aad) if aad_len else None
    out, ok = aes.gcm_open(dev(ct), ks, iv, dev(tag), aad=d_aad)
    assert int(host(ok)[0]) == 1 and (host(out) == pt).all()
    # any wrong tag byte, ciphertext bit or AAD byte fails the check
    for b in (0, 7, 15):
        bad = tag.copy()
        bad[b] ^= 0x40
        _, ok = aes.gcm_open(dev(ct), ks, iv, dev(bad), aad=d_aad)
        assert int(host(ok)[0]) == 0, b
    if nbytes:
        ct2 = ct.copy()
        ct2[nbytes // 2] ^= 1
        _, ok = aes.gcm_open(dev(ct2), ks, iv, dev(tag), aad=d_aad)
        assert int(host(ok)[0]) == 0
    if aad_len:
        aad2 = aad.copy()
        aad2[0] ^= 0x80
        _, ok = aes.gcm_open(dev(ct), ks, iv, dev(tag), aad=dev(aad2))
        assert int(host(ok)[0]) == 0
    # in place
    x = dev(ct)
    _, ok = aes.gcm_open(x, ks, iv, dev(tag), aad=d_aad, out=x)
    assert int(host(ok)[0]) == 1 and (host(x) == pt).all()


@pytest.mark.parametrize("nb", [1, 2, 3, 31, 32, 33, 64, 65, 128, 129, 152])
def test_gcm_every_cross_cta_tree_depth(aes, orc, cuda, nb):
    """The CTA that finishes last combines the CTAs' partial sums with a tree of as many levels
    as the CTA count needs (none for one CTA, up to eight): hashed-block counts that give each
    count of CTAs (512 positions per CTA) around the powers of two."""
    n = 512 * (nb - 1) + 1 + (nb % 7) * 11
    rng = np.random.default_rng(500 + nb)
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    iv = rng.integers(0, 256, 12, dtype=np.uint8)
    pt = rng.integers(0, 256, 16 * (n - 1) + 5, dtype=np.uint8)  # n blocks, the last ragged
    ks = aes.aes_key_expand(key.tobytes())
    want_ct, want_tag = orc.gcm_crypt(key, iv, pt)
    ct, tag = aes.gcm(dev(pt), ks, iv.tobytes())
    assert (host(tag) == want_tag).all()
    assert (host(ct) == want_ct).all()


def test_gcm_iv_length_limits(aes, cuda):
    import torch

    ks = aes.aes_key_expand(bytes(16))
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for bad in (b"", bytes(257)):
        with pytest.raises(aes.AesError):
            aes.gcm(x, ks, bad)


def test_gcm_decrypt_of_arbitrary_data_and_in_place(aes, orc, cuda):
    rng = np.random.default_rng(9)
    key, iv = rng.integers(0, 256, 32, dtype=np.uint8), rng.integers(0, 256, 12, dtype=np.uint8)
    data, aad = rng.integers(0, 256, 16 * 50_001 + 7, dtype=np.uint8), rng.integers(0, 256, 40, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), 256)
    want, want_tag = orc.gcm_crypt(key, iv, data, aad, decrypt=True)
    x = dev(data)
    _, tag = aes.gcm(x, ks, iv.tobytes(), aad=dev(aad), dir="decrypt", out=x)
    assert (host(x) == want).all() and (host(tag) == want_tag).all()


def test_gcm_calls_in_a_row_share_nothing(aes, orc, cuda):
    # different keys, IVs and sizes back to back on one stream, each with a fresh workspace
    rng = np.random.default_rng(10)
    outs = []
    for n in (5000, 16, 16 * 300_000):
        key, iv = rng.integers(0, 256, 16, dtype=np.uint8), rng.integers(0, 256, 12, dtype=np.uint8)
        pt = rng.integers(0, 256, n, dtype=np.uint8)
        ct, tag = aes.gcm(dev(pt), aes.aes_key_expand(key.tobytes()), iv.tobytes())
        outs.append((key, iv, pt, ct, tag))
    for key, iv, pt, ct, tag in outs:
        want_ct, want_tag = orc.gcm_crypt(key, iv, pt)
        assert (host(ct) == want_ct).all() and (host(tag) == want_tag).all()


def _power(orc, h, e):
    acc = np.array([0x80] + [0] * 15, dtype=np.uint8)
    sq = h.copy()
    while e:
        if e & 1:
            acc = orc.gf128_mul(acc, sq)
        sq = orc.gf128_mul(sq, sq)
        e >>= 1
    return acc


def test_gcm_full_size_1gib(aes, orc, cuda):
    """2^26 blocks (1 GiB): the bench's GCM workload and launch."""
    import torch

    c = 1 << 26
    rng = np.random.default_rng(11)
    key, iv = rng.integers(0, 256, 16, dtype=np.uint8), rng.integers(0, 256, 12, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes())
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randint(0, 256, (16 * c,), dtype=torch.uint8, device="cuda", generator=g)
    ct, tag = aes.gcm(x, ks, iv.tobytes())
    # sampled blocks: C_j = P_j + Cipher(IV || 2 + j)
    idx = np.unique(np.concatenate([[0, 1, c // 2, c - 2, c - 1], rng.integers(0, c, 2000)]))
    ti = torch.from_numpy(idx).cuda()
    p = x.view(-1, 16)[ti].cpu().numpy()
    got = ct.view(-1, 16)[ti].cpu().numpy()
    ctrs = np.zeros((idx.size, 16), dtype=np.uint8)
    ctrs[:, :12] = iv
    ctrs[:, 12:] = np.frombuffer(b"".join(int(2 + j).to_bytes(4, "big") for j in idx), dtype=np.uint8).reshape(-1, 4)
    ks_blocks = orc.encrypt_blocks(key, ctrs.reshape(-1), threads=8).reshape(-1, 16)
    assert (got == (p ^ ks_blocks)).all()
    # decryption returns the plaintext and the same tag
    back, tag2 = aes.gcm(ct, ks, iv.tobytes(), dir="decrypt")
    torch.cuda.synchronize()
    assert torch.equal(back, x) and torch.equal(tag, tag2)
    del back, ct
    # sparse ciphertext: the tag has a closed form in H
    h = orc.encrypt_blocks(key, np.zeros(16, dtype=np.uint8))
    ej0 = orc.encrypt_blocks(key, np.concatenate([iv, np.array([0, 0, 0, 1], dtype=np.uint8)]))
    x.zero_()
    pos = [0, 1, 77_823, 77_824, c // 3, c - 2, c - 1]
    vals = rng.integers(0, 256, (len(pos), 16), dtype=np.uint8)
    x.view(-1, 16)[torch.tensor(pos, device="cuda")] = torch.from_numpy(vals).cuda()
    _, tag3 = aes.gcm(x, ks, iv.tobytes(), dir="decrypt")
    s = np.zeros(16, dtype=np.uint8)
    for j, v in zip(pos, vals):
        s ^= orc.gf128_mul(v, _power(orc, h, c - j + 1))
    lens = np.frombuffer((0).to_bytes(8, "big") + (128 * c).to_bytes(8, "big"), dtype=np.uint8)
    s ^= orc.gf128_mul(lens, h)
    assert (host(tag3) == (ej0 ^ s)).all()
    del x
    torch.cuda.empty_cache()


def test_gcm_beyond_4gib(aes, orc, cuda):
    """2^28 + 1027 blocks (just over 4 GiB): positions, counters and GHASH exponents past 2^28
    blocks and byte offsets past 2^32.  A sparse ciphertext gives a closed-form tag; sampled
    blocks on both sides of 2^28 are checked against the oracle's cipher of their counters."""
    import torch

    c = (1 << 28) + 1027
    rng = np.random.default_rng(12)
    key, iv = rng.integers(0, 256, 16, dtype=np.uint8), rng.integers(0, 256, 12, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes())
    x = torch.zeros(16 * c, dtype=torch.uint8, device="cuda")
    pos = [0, 77_823, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, c - 1]
    vals = rng.integers(0, 256, (len(pos), 16), dtype=np.uint8)
    x.view(-1, 16)[torch.tensor(pos, device="cuda")] = torch.from_numpy(vals).cuda()
    aad = torch.from_numpy(rng.integers(0, 256, 20, dtype=np.uint8)).cuda()
    out, tag = aes.gcm(x, ks, iv.tobytes(), aad=aad, dir="decrypt")
    h = orc.encrypt_blocks(key, np.zeros(16, dtype=np.uint8))
    ej0 = orc.encrypt_blocks(key, np.concatenate([iv, np.array([0, 0, 0, 1], dtype=np.uint8)]))
    a_host = aad.cpu().numpy()
    a_blocks = np.zeros(32, dtype=np.uint8)
    a_blocks[:20] = a_host
    m = 2 + c + 1  # AAD blocks, data blocks, length block
    s = orc.gf128_mul(a_blocks[:16], _power(orc, h, m)) ^ orc.gf128_mul(a_blocks[16:], _power(orc, h, m - 1))
    for j, v in zip(pos, vals):
        s ^= orc.gf128_mul(v, _power(orc, h, c - j + 1))
    lens = np.frombuffer((160).to_bytes(8, "big") + (128 * c).to_bytes(8, "big"), dtype=np.uint8)
    s ^= orc.gf128_mul(lens, h)
    assert (tag.cpu().numpy() == (ej0 ^ s)).all()
    # keystream blocks: out_j = x_j + Cipher(IV || 2 + j)
    idx = np.array(pos + [12345, (1 << 28) + 700], dtype=np.int64)
    got = out.view(-1, 16)[torch.from_numpy(idx).cuda()].cpu().numpy()
    src = x.view(-1, 16)[torch.from_numpy(idx).cuda()].cpu().numpy()
    ctrs = np.zeros((idx.size, 16), dtype=np.uint8)
    ctrs[:, :12] = iv
    ctrs[:, 12:] = np.frombuffer(b"".join(int(2 + j).to_bytes(4, "big") for j in idx), dtype=np.uint8).reshape(-1, 4)
    ksb = orc.encrypt_blocks(key, ctrs.reshape(-1)).reshape(-1, 16)
    assert (got == (src ^ ksb)).all()
    del x, out
    torch.cuda.empty_cache()
