"""GPU parity of the paper's CBC mode over whole messages (Section II; App. A1, A4) against
the oracle's per-message CBC (itself pinned to OpenSSL CBC).  Bit-exact."""
import os

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("key_bits", [128, 192, 256])
@pytest.mark.parametrize("m", [1, 2, 17, 100])
def test_paper_shape_128_messages_one_iv(aes_lib_ready, orc, key_bits, m):
    # the paper's second workload shape: 128 messages of a given length, one repeated IV
    rng = np.random.default_rng(70 + m + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    iv = rng.integers(0, 256, 16, dtype=np.uint8)
    pt = rng.integers(0, 256, (128, 16 * m), dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    ct = aes.cbc(dev(pt), ks, dev(iv), "encrypt").cpu().numpy()
    for i in range(128):
        assert (ct[i] == orc.cbc_encrypt(key, iv, pt[i])).all(), i
    back = aes.cbc(dev(ct), ks, dev(iv), "decrypt").cpu().numpy()
    assert (back == pt).all()


def test_iv_per_message_and_many_messages(aes_lib_ready, orc):
    rng = np.random.default_rng(80)
    n, m = 20011, 9
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    pt = rng.integers(0, 256, (n, 16 * m), dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes())
    ct = aes.cbc(dev(pt), ks, dev(ivs), "encrypt").cpu().numpy()
    for i in list(range(0, n, 997)) + [n - 1]:
        assert (ct[i] == orc.cbc_encrypt(key, ivs[i], pt[i])).all(), i
    # decryption of arbitrary data matches the oracle too (not only round trips)
    junk = rng.integers(0, 256, (n, 16 * m), dtype=np.uint8)
    dj = aes.cbc(dev(junk), ks, dev(ivs), "decrypt").cpu().numpy()
    for i in list(range(0, n, 1999)) + [n - 1]:
        assert (dj[i] == orc.cbc_decrypt(key, ivs[i], junk[i])).all(), i
    assert (aes.cbc(dev(ct), ks, dev(ivs), "decrypt").cpu().numpy() == pt).all()


def test_long_single_message_and_in_place(aes_lib_ready, orc):
    import torch

    rng = np.random.default_rng(81)
    key = rng.integers(0, 256, 32, dtype=np.uint8)
    iv = rng.integers(0, 256, 16, dtype=np.uint8)
    pt = rng.integers(0, 256, (1, 16 * 5000), dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), 256)
    x = dev(pt)
    aes.cbc(x, ks, dev(iv), "encrypt", out=x)  # encryption may run in place
    torch.cuda.synchronize()
    assert (x.cpu().numpy()[0] == orc.cbc_encrypt(key, iv, pt[0])).all()
    with pytest.raises(aes.AesError) as ei:
        aes.cbc(x, ks, dev(iv), "decrypt", out=x)
    assert ei.value.status == aes.AES_EINVAL
    y = aes.cbc(x, ks, dev(iv), "decrypt")
    assert (y.cpu().numpy() == pt).all()


def test_cbc_argument_checks(aes_lib_ready):
    import torch

    ks = aes.aes_key_expand(bytes(16))
    x = torch.zeros((4, 64), dtype=torch.uint8, device="cuda")
    iv = torch.zeros(16, dtype=torch.uint8, device="cuda")
    lib = aes.lib()
    import ctypes

    assert lib.aes_cbc_crypt(ctypes.byref(ks), iv.data_ptr(), 0, x.data_ptr(), x.data_ptr(), 0, 4, 0, None) == 0
    assert lib.aes_cbc_crypt(ctypes.byref(ks), iv.data_ptr(), 2, x.data_ptr(), x.data_ptr(), 4, 4, 0, None) == aes.AES_EINVAL
    assert lib.aes_cbc_crypt(ctypes.byref(ks), iv.data_ptr() + 8, 0, x.data_ptr(), x.data_ptr(), 4, 4, 0, None) == aes.AES_EINVAL
    assert lib.aes_cbc_crypt(ctypes.byref(ks), None, 0, x.data_ptr(), x.data_ptr(), 4, 4, 0, None) == aes.AES_EINVAL
    assert lib.aes_cbc_crypt(ctypes.byref(ks), iv.data_ptr(), 0, x.data_ptr(), x.data_ptr() + 16, 4, 4, 0, None) == aes.AES_EINVAL


def test_bench_shape_2p18_messages_sampled(aes_lib_ready, orc):
    """2^18 messages x 16 blocks (64 MiB), one IV per message: the benchmark's CBC row, in the
    launch the benchmark times; sampled messages against the oracle, full round trip."""
    import torch

    n, m = 1 << 18, 16
    g = torch.Generator(device="cuda").manual_seed(82)
    x = torch.randint(0, 256, (n, 16 * m), dtype=torch.uint8, device="cuda", generator=g)
    ivs = torch.randint(0, 256, (n, 16), dtype=torch.uint8, device="cuda", generator=g)
    key = np.arange(16, dtype=np.uint8) * 11
    ks = aes.aes_key_expand(key.tobytes())
    ct = aes.cbc(x, ks, ivs, "encrypt")
    rows = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], np.random.default_rng(83).integers(0, n, 300)]))
    tr = torch.from_numpy(rows).cuda()
    p, c, v = x[tr].cpu().numpy(), ct[tr].cpu().numpy(), ivs[tr].cpu().numpy()
    for k in range(rows.size):
        assert (c[k] == orc.cbc_encrypt(key, v[k], p[k])).all(), rows[k]
    back = aes.cbc(ct, ks, ivs, "decrypt")
    torch.cuda.synchronize()
    assert torch.equal(back, x)


@pytest.mark.parametrize("m", [1, 13, 16, 21])
def test_staged_encrypt_ragged(aes_lib_ready, orc, m):
    """Enough messages for the staged (shared-memory tiled) encryption kernel, a message count
    that leaves the last warp's group partial, and lengths that leave the last stage partial."""
    import torch

    n = 160_037  # above the staged kernel's threshold (one group of 32 per warp of a full GPU)
    g = torch.Generator(device="cuda").manual_seed(84 + m)
    x = torch.randint(0, 256, (n, 16 * m), dtype=torch.uint8, device="cuda", generator=g)
    ivs = torch.randint(0, 256, (n, 16), dtype=torch.uint8, device="cuda", generator=g)
    key = np.arange(32, dtype=np.uint8) * 5
    ks = aes.aes_key_expand(key.tobytes(), 256)
    ct = aes.cbc(x, ks, ivs, "encrypt")
    rows = np.unique(np.concatenate([np.arange(0, 40), np.arange(n - 40, n),
                                     np.random.default_rng(85).integers(0, n, 200)]))
    tr = torch.from_numpy(rows).cuda()
    p, c, v = x[tr].cpu().numpy(), ct[tr].cpu().numpy(), ivs[tr].cpu().numpy()
    for k in range(rows.size):
        assert (c[k] == orc.cbc_encrypt(key, v[k], p[k])).all(), rows[k]
    y = x.clone()
    aes.cbc(y, ks, ivs, "encrypt", out=y)  # in place
    torch.cuda.synchronize()
    assert torch.equal(y, ct)
    assert torch.equal(aes.cbc(ct, ks, ivs, "decrypt"), x)


@pytest.mark.parametrize("n", [97_280, 97_307, 160_037])
def test_staged_encrypt_each_cta_size(aes_lib_ready, orc, n):
    """The staged kernel's CTA size follows the number of 32-message groups (the fewest waves
    over the SMs).  On a 152-SM GPU these counts take 20, 16 and 18 warps per CTA: 3040 groups
    (one full wave of 20 warps), 3041 groups (two waves at every size, so the smallest), and
    5002 groups (two waves of 18 or 20 warps).  AES-192 and one IV for all messages."""
    import torch

    m = 5
    g = torch.Generator(device="cuda").manual_seed(86)
    x = torch.randint(0, 256, (n, 16 * m), dtype=torch.uint8, device="cuda", generator=g)
    iv = torch.randint(0, 256, (16,), dtype=torch.uint8, device="cuda", generator=g)
    key = (np.arange(24, dtype=np.uint8) * 7 + 3).astype(np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), 192)
    ct = aes.cbc(x, ks, iv, "encrypt")
    rows = np.unique(np.concatenate([np.arange(0, 33), np.arange(n - 33, n),
                                     np.random.default_rng(87).integers(0, n, 150)]))
    tr = torch.from_numpy(rows).cuda()
    p, c, v = x[tr].cpu().numpy(), ct[tr].cpu().numpy(), iv.cpu().numpy()
    for k in range(rows.size):
        assert (c[k] == orc.cbc_encrypt(key, v, p[k])).all(), rows[k]
    assert torch.equal(aes.cbc(ct, ks, iv, "decrypt"), x)


def _sms():
    import torch

    return torch.cuda.get_device_properties(0).multi_processor_count


# message counts that reach every launch shape of the four-lanes-per-chain encryption (per SM:
# up to 4 chains one per warp, up to 32 on four warps, up to 64 at eight chains per warp) and
# the one-lane kernel just past it: per-SM counts times the device's SM count, plus ragged ones
CHAINS_PER_SM = [(0, 1), (0, 129), (4, 0), (4, 1), (20, 7), (32, 0), (32, 1), (64, 0), (64, 1)]


@pytest.mark.parametrize("per_sm,extra", CHAINS_PER_SM, ids=[f"{a}xSM+{b}" for a, b in CHAINS_PER_SM])
def test_encrypt_chain_shapes(aes_lib_ready, orc, per_sm, extra):
    """CBC encryption at every chains-per-warp shape: sampled messages (first, last and 150
    random ones, each with its own IV) against the oracle, then the whole matrix round trip."""
    import torch

    n, m = per_sm * _sms() + extra, 3
    rng = np.random.default_rng(84 + n)
    key = rng.integers(0, 256, 32 if per_sm == 20 else 16, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), 8 * key.size)
    pt = rng.integers(0, 256, (n, 16 * m), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    x = dev(pt)
    ct = aes.cbc(x, ks, dev(ivs), "encrypt").cpu().numpy()
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 150)]))
    for i in rows:
        assert (ct[i] == orc.cbc_encrypt(key, ivs[i], pt[i])).all(), i
    back = aes.cbc(dev(ct), ks, dev(ivs), "decrypt")
    torch.cuda.synchronize()
    assert torch.equal(back, x)


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (128, 16), (128, 256), (257, 128), (129, 255)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("key_bits", [128, 256])
def test_decrypt_small_matrices(aes_lib_ready, orc, shape, key_bits):
    """Decryption of arbitrary data (not only round trips) of small matrices, down to a single
    block, and of a few thousand blocks up to 32896, with one IV per message and with one
    shared IV, against the oracle's CBC."""
    n, m = shape
    rng = np.random.default_rng(90 + n * 7 + m + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    ct = rng.integers(0, 256, (n, 16 * m), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    for iv_arg, iv_of in ((ivs, lambda i: ivs[i]), (ivs[0], lambda i: ivs[0])):
        pt = aes.cbc(dev(ct), ks, dev(iv_arg), "decrypt").cpu().numpy()
        rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 40)]))
        for i in rows:
            assert (pt[i] == orc.cbc_decrypt(key, iv_of(i), ct[i])).all(), (i, iv_arg.ndim)
