"""GPU parity: the CUDA kernels, called through the C ABI, against the CPU oracle.

Every comparison is bit-exact (the arithmetic is integer).  Small and ragged sizes are
compared element by element over the whole buffer; the full-size workloads (1 GiB of
blocks, 10^7 sensor records) are compared on sampled blocks that the oracle computes one by
one, plus a full decrypt(encrypt(x)) == x round trip on the device.
"""
import os

import numpy as np
import pytest

from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
IMPLS = ["ttable", "bitslice"]


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t) -> np.ndarray:
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def run(aes, ks, x, direction, impl, iv=None, out=None):
    return aes.crypt(x, ks, direction, iv=iv, out=out, impl=impl)


@pytest.mark.parametrize("impl", IMPLS)
def test_plain_4096_blocks_seed0(aes, orc, cuda, impl):
    w = workloads.plain(0, 4096)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = to_dev(w.data)
    ct = run(aes, ks, x, "encrypt", impl)
    want = orc.encrypt_blocks(w.key, w.data, threads=THREADS)
    assert (to_host(ct) == want).all()
    pt = run(aes, ks, ct, "decrypt", impl)
    assert (to_host(pt) == w.data).all()
    assert (orc.decrypt_blocks(w.key, want, threads=THREADS) == w.data).all()


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 511, 513, 1023, 1025, 4097, 77_825, 155_651])
def test_ragged_sizes(aes, orc, cuda, impl, n):
    w = workloads.plain(100 + n, n)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = to_dev(w.data)
    ct = to_host(run(aes, ks, x, "encrypt", impl))
    assert (ct == orc.encrypt_blocks(w.key, w.data, threads=THREADS)).all()
    pt = to_host(run(aes, ks, to_dev(ct), "decrypt", impl))
    assert (pt == w.data).all()


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("key_bits", [128, 192, 256])
def test_key_sizes_and_iv(aes, orc, cuda, impl, key_bits):
    rng = np.random.default_rng(key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    iv = rng.integers(0, 256, 16, dtype=np.uint8)
    data = rng.integers(0, 256, 16 * 20_011, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    ct = to_host(run(aes, ks, to_dev(data), "encrypt", impl, iv=iv.tobytes()))
    assert (ct == orc.encrypt_blocks(key, data, iv=iv, threads=THREADS)).all()
    pt = to_host(run(aes, ks, to_dev(ct), "decrypt", impl, iv=iv.tobytes()))
    assert (pt == data).all()
    # decryption of arbitrary data (not produced by encryption) also matches
    dd = to_host(run(aes, ks, to_dev(data), "decrypt", impl, iv=iv.tobytes()))
    assert (dd == orc.decrypt_blocks(key, data, iv=iv, threads=THREADS)).all()


@pytest.mark.parametrize("impl", IMPLS)
def test_in_place(aes, orc, cuda, impl):
    w = workloads.plain(7, 50_003)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = to_dev(w.data)
    aes.crypt(x, ks, "encrypt", out=x, impl=impl)
    assert (to_host(x) == orc.encrypt_blocks(w.key, w.data, threads=THREADS)).all()
    aes.crypt(x, ks, "decrypt", out=x, impl=impl)
    assert (to_host(x) == w.data).all()


def test_impls_agree_and_auto(aes, cuda):
    import torch

    w = workloads.plain(9, 300_007)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = to_dev(w.data)
    a = aes.encrypt(x, ks, impl="ttable")
    b = aes.encrypt(x, ks, impl="bitslice")
    c = aes.encrypt(x, ks)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("key_bits", [128, 192, 256])
def test_small_call_kernel(aes, orc, cuda, key_bits):
    """AES_IMPL_AUTO calls of up to 32768 blocks run the small-call kernel (tables read from
    global memory, no shared-memory fill): ragged sizes up to the threshold, with and without
    IV, both directions, against the oracle; one block past the threshold takes the other
    kernel and agrees."""
    import torch

    for d in ("encrypt", "decrypt"):
        aes.aes_set_auto_choice(d, {128: 10, 192: 12, 256: 14}[key_bits], "auto", 0, 0)  # no pinned choice
    rng = np.random.default_rng(500 + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    for n in (1, 2, 31, 127, 129, 4096, 4097, 32768, 32769):
        for iv in (None, rng.integers(0, 256, 16, dtype=np.uint8)):
            data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
            x = to_dev(data)
            ivb = None if iv is None else iv.tobytes()
            ct = to_host(aes.encrypt(x, ks, iv=ivb))
            assert (ct == orc.encrypt_blocks(key, data, iv=iv, threads=THREADS)).all(), n
            dd = to_host(aes.decrypt(x, ks, iv=ivb))
            assert (dd == orc.decrypt_blocks(key, data, iv=iv, threads=THREADS)).all(), n


def test_empty_is_noop(aes, cuda):
    import torch

    ks = aes.aes_key_expand(bytes(16))
    x = torch.zeros(0, dtype=torch.uint8, device="cuda")
    aes.encrypt(x, ks)


def _sampled_check(orc, key, host_in, dev_out, idx, iv=None, decrypt=False):
    import torch

    torch.cuda.synchronize()
    got = dev_out.view(-1, 16)[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1)
    src = host_in.reshape(-1, 16)[idx].reshape(-1)
    want = (orc.decrypt_blocks if decrypt else orc.encrypt_blocks)(key, src, iv=iv, threads=THREADS)
    assert (got == want).all()


def _sample_idx(n: int, seed: int, k: int = 20_000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    edge = np.array([0, 1, 2, n // 2, n - 3, n - 2, n - 1], dtype=np.int64)
    return np.unique(np.concatenate([edge, rng.integers(0, n, size=k)]))


@pytest.mark.parametrize("impl", IMPLS)
def test_full_size_1gib(aes, orc, cuda, impl):
    """2^26 blocks (1 GiB) of seed-1 random bytes, the benchmark's workload and launch."""
    import torch

    n = 1 << 26
    w = workloads.plain(1, n)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = to_dev(w.data)
    ct = aes.encrypt(x, ks, impl=impl)
    idx = _sample_idx(n, 1)
    _sampled_check(orc, w.key, w.data, ct, idx)
    pt = aes.decrypt(ct, ks, impl=impl)
    torch.cuda.synchronize()
    assert torch.equal(pt, x)
    del ct, pt, x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("key_name", ["key128", "key256"])
def test_sensor_records(aes, orc, cuda, key_name):
    """10^7 16-byte records (int64 timestamp, int64 Gaussian reading), AES-128 and AES-256."""
    import torch

    col = workloads.sensor_records(2, 10_000_000)
    key = getattr(col, key_name)
    ks = aes.aes_key_expand(key.tobytes())
    x = to_dev(col.records)
    ct = aes.encrypt(x, ks)
    _sampled_check(orc, key, col.records, ct, _sample_idx(10_000_000, 2))
    pt = aes.decrypt(ct, ks)
    torch.cuda.synchronize()
    assert torch.equal(pt, x)


def test_buffer_beyond_4gib(aes, orc, cuda):
    """2^28 + 1027 blocks (just over 4 GiB): block indices pass 2^28 and byte offsets pass 2^32,
    so 32-bit index arithmetic anywhere would show.  Plain, batched and counter-mode paths."""
    import torch

    n = (1 << 28) + 1027
    g = torch.Generator(device="cuda").manual_seed(28)
    x = torch.randint(0, 256, (n * 16,), dtype=torch.uint8, device="cuda", generator=g)
    key = np.arange(16, dtype=np.uint8) * 7
    ks = aes.aes_key_expand(key.tobytes())
    idx = np.array([0, 1, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, n - 2, n - 1] +
                   list(np.random.default_rng(3).integers(0, n, 64)), dtype=np.int64)
    ti = torch.from_numpy(idx).cuda()
    before = x.view(-1, 16)[ti].cpu().numpy().reshape(-1)
    aes.encrypt(x, ks, out=x)  # in place: 4 GiB is enough memory for this test
    got = x.view(-1, 16)[ti].cpu().numpy().reshape(-1)
    assert (got == orc.encrypt_blocks(key, before, threads=THREADS)).all()
    aes.decrypt(x, ks, out=x)
    assert (x.view(-1, 16)[ti].cpu().numpy().reshape(-1) == before).all()
    # batched: messages placed past the 4 GiB mark, each with its own key
    with aes.KeyPool(3) as pool:
        keys = np.stack([key, key[::-1].copy(), key ^ 0x5A])
        pool.load_keys(0, keys, 128)
        # the buffer ends 1027 blocks past 2^32 bytes; the three messages do not overlap
        offs = [(1 << 32) - 16 * 5, (1 << 32) + 16 * 10, 16 * (n - 300)]
        msgs = np.zeros(3, dtype=aes.msg_dtype())
        msgs["key_idx"], msgs["offset"], msgs["length"] = [0, 1, 2], offs, [16 * 10, 16 * 700, 16 * 300]
        src = [x[o:o + int(L)].cpu().numpy() for o, L in zip(offs, msgs["length"])]
        aes.aes_crypt_batched(pool, msgs, x.data_ptr(), x.data_ptr(), n * 16)
        torch.cuda.synchronize()
        for k, (o, L) in enumerate(zip(offs, msgs["length"])):
            assert (x[o:o + int(L)].cpu().numpy() == orc.encrypt_blocks(keys[k], src[k], threads=THREADS)).all()
    # counter mode over the whole buffer: blocks past index 2^28 use counters past 2^28
    ctr0 = bytes(16)
    before = x.view(-1, 16)[ti].cpu().numpy()
    aes.ctr(x, ks, ctr0, out=x)
    got = x.view(-1, 16)[ti].cpu().numpy()
    for j, i in enumerate(idx):
        c = int(i).to_bytes(16, "big")
        ksb = orc.encrypt_blocks(key, np.frombuffer(c, dtype=np.uint8))
        assert (got[j] == (before[j] ^ ksb)).all(), i
    del x
    torch.cuda.empty_cache()
