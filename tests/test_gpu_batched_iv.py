"""GPU parity of the batched paths with one IV per message (the IV matrix V of the paper's
Section II, one row per message, with the key tensor K's schedule per message), through the C
ABI, against the CPU oracle, bit-exact, message by message:
  * aes_crypt_batched_iv / aes_batch_run_iv: every block of message i is a one-block CBC
    message, C = Cipher_Ki(P ^ IV_i), and decryption P = InvCipher_Ki(C) ^ IV_i;
  * aes_cbc_batched: the paper's CBC chained over each whole message (App. A1/A4),
    C_j = Cipher_Ki(P_j ^ C_{j-1}) with C_{-1} = IV_i.
"""
import os

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes
from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _expect(orc, keys, key_idx, dirs, ivs, offsets, lengths, data):
    out = data.copy()
    for i in range(len(lengths)):
        o, L = int(offsets[i]), int(lengths[i])
        if not L:
            continue
        f = orc.decrypt_blocks if dirs[i] else orc.encrypt_blocks
        out[o:o + L] = f(keys[int(key_idx[i])], data[o:o + L], iv=ivs[i], threads=THREADS)
    return out


def test_4096_lognormal_messages_own_key_and_iv(aes_lib_ready, orc):
    """The batched workload (4096 lognormal messages, seed 3, own AES-128 key each) with a random
    IV per message: encryption against the oracle on every message, then decryption back."""
    import torch

    m = workloads.batched_messages(3)
    n = len(m.lengths)
    ivs = np.random.default_rng(70).integers(0, 256, (n, 16), dtype=np.uint8)
    total = int(m.lengths.sum())
    with aes.KeyPool(n) as pool:
        pool.load_keys(0, m.keys, 128)
        msgs = np.zeros(n, dtype=aes.msg_dtype())
        msgs["key_idx"] = np.arange(n)
        msgs["offset"], msgs["length"] = m.offsets, m.lengths
        x = dev(m.data)
        y = torch.empty_like(x)
        aes.aes_crypt_batched_iv(pool, msgs, ivs, x.data_ptr(), y.data_ptr(), total)
        want = _expect(orc, list(m.keys), np.arange(n), np.zeros(n, dtype=np.uint32), ivs, m.offsets, m.lengths,
                       m.data)
        assert np.array_equal(host(y), want)
        msgs["dir"] = 1
        z = torch.empty_like(x)
        aes.aes_crypt_batched_iv(pool, msgs, ivs, y.data_ptr(), z.data_ptr(), total)
        assert torch.equal(z, x)
        # without IVs the same call is aes_crypt_batched (zero IVs)
        aes.aes_crypt_batched(pool, msgs, y.data_ptr(), z.data_ptr(), total)
        w = torch.empty_like(x)
        aes.aes_crypt_batched_iv(pool, msgs, np.zeros((n, 16), dtype=np.uint8), y.data_ptr(), w.data_ptr(), total)
        torch.cuda.synchronize()
        assert torch.equal(z, w)


@pytest.mark.parametrize("shape", [(512, 1), (512, 2), (512, 4), (384, 4), (256, 4), (768, 1)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_shared_keys_mixed_sizes_both_directions(aes_lib_ready, orc, shape):
    """Few keys shared by many messages (so a warp changes message without changing key and
    swaps only the IV), AES-128/192/256 keys, both directions in one launch, empty messages,
    at every compiled shape (768 x 1 with AES-128 keys only)."""
    import torch

    rng = np.random.default_rng(71 + shape[0] + shape[1])
    n = 600
    aes128_only = shape == (768, 1)
    bits = [128] * 6 if aes128_only else [128, 128, 192, 256, 256, 128]
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8) for b in bits]
    key_idx = rng.integers(0, len(keys), n).astype(np.uint32)
    dirs = rng.integers(0, 2, n).astype(np.uint32)
    lengths = (rng.integers(0, 90, n) * 16).astype(np.int64)
    lengths[::23] = 0
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["dir"], msgs["offset"], msgs["length"] = key_idx, dirs, offsets, lengths
    want = _expect(orc, keys, key_idx, dirs, ivs, offsets, lengths, data)
    with aes.KeyPool(len(keys)) as pool:
        for i, k in enumerate(keys):
            pool.set(i, aes.aes_key_expand(k.tobytes(), 8 * len(k)))
        with aes.Batch(pool, n) as b:
            b.set_shape(*shape)
            x = dev(data)
            for _ in range(2):  # the second run replays the cached graph
                y = x.clone()
                b.run(msgs, x.data_ptr(), y.data_ptr(), data.size, ivs=ivs)
                assert np.array_equal(host(y), want)
            # in place
            b.run(msgs, x.data_ptr(), x.data_ptr(), data.size, ivs=ivs)
            assert np.array_equal(host(x), want)


def test_iv_array_size_is_checked(aes_lib_ready):
    with aes.KeyPool(1) as pool:
        pool.set(0, aes.aes_key_expand(bytes(16)))
        msgs = np.zeros(2, dtype=aes.msg_dtype())
        with pytest.raises(ValueError):
            aes.aes_crypt_batched_iv(pool, msgs, np.zeros(16, dtype=np.uint8), 0, 0, 0)


def _cbc_expect(orc, keys, key_idx, dirs, ivs, offsets, lengths, data):
    out = data.copy()
    for i in range(len(lengths)):
        o, L = int(offsets[i]), int(lengths[i])
        if not L:
            continue
        iv = ivs[i] if ivs is not None else np.zeros(16, np.uint8)
        f = orc.cbc_decrypt if dirs[i] else orc.cbc_encrypt
        out[o:o + L] = f(keys[int(key_idx[i])], iv, data[o:o + L])
    return out


@pytest.mark.parametrize("with_ivs", [True, False])
def test_cbc_chained_messages_own_keys_and_ivs(aes_lib_ready, orc, with_ivs):
    """The paper's CBC over whole messages in its general form (aes_cbc_batched): lognormal
    lengths, AES-128/192/256 keys, each message with its own key and IV, both directions in one
    call, empty messages; every message against the oracle's CBC, and decryption of the
    ciphertext restores the plaintext."""
    import torch

    rng = np.random.default_rng(80 + with_ivs)
    n = 400
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8) for b in (128, 192, 256) for _ in range(5)]
    key_idx = rng.integers(0, len(keys), n).astype(np.uint32)
    dirs = rng.integers(0, 2, n).astype(np.uint32)
    m = workloads.batched_messages(81, m=n, median=512.0, hi=1 << 16)
    lengths = m.lengths.copy()
    lengths[::37] = 0
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8) if with_ivs else None
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["dir"], msgs["offset"], msgs["length"] = key_idx, dirs, m.offsets, lengths
    want = _cbc_expect(orc, keys, key_idx, dirs, ivs, m.offsets, lengths, m.data)
    with aes.KeyPool(len(keys)) as pool:
        for i, k in enumerate(keys):
            pool.load_keys(i, k[None, :], 8 * len(k))
        x = dev(m.data)
        y = x.clone()
        aes.aes_cbc_batched(pool, msgs, ivs, x.data_ptr(), y.data_ptr(), m.data.size)
        assert np.array_equal(host(y), want)
        # the encrypted messages decrypt back (all messages decrypted this time)
        enc = msgs["dir"] == 0
        back = msgs.copy()
        back["dir"] = 1
        back["length"] = np.where(enc, msgs["length"], 0)
        z = y.clone()
        aes.aes_cbc_batched(pool, back, ivs, y.data_ptr(), z.data_ptr(), m.data.size)
        zz = host(z)
        for i in np.nonzero(enc & (lengths > 0))[0]:
            o, L = int(m.offsets[i]), int(lengths[i])
            assert np.array_equal(zz[o:o + L], m.data[o:o + L]), i


def test_cbc_128_messages_of_varying_length(aes_lib_ready, orc):
    """The paper's second workload shape (Section IV, Fig. 3): 128 messages of lengths from one
    block to 4096 blocks, one AES-128 key and IV each, encrypted and decrypted."""
    import torch

    rng = np.random.default_rng(82)
    n = 128
    lengths = (np.unique(np.geomspace(1, 4096, n).astype(np.int64), return_counts=False))
    lengths = np.resize(lengths, n) * 16
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    keys = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["offset"], msgs["length"] = np.arange(n), offsets, lengths
    with aes.KeyPool(n) as pool:
        pool.load_keys(0, keys, 128)
        x = dev(data)
        y = torch.empty_like(x)
        aes.aes_cbc_batched(pool, msgs, ivs, x.data_ptr(), y.data_ptr(), data.size)
        ct = host(y)
        for i in range(n):
            o, L = int(offsets[i]), int(lengths[i])
            assert np.array_equal(ct[o:o + L], orc.cbc_encrypt(keys[i], ivs[i], data[o:o + L])), i
        msgs["dir"] = 1
        z = torch.empty_like(x)
        aes.aes_cbc_batched(pool, msgs, ivs, y.data_ptr(), z.data_ptr(), data.size)
        assert torch.equal(z, x)
        with pytest.raises(aes.AesError):  # decryption in place is refused
            aes.aes_cbc_batched(pool, msgs, ivs, y.data_ptr(), y.data_ptr(), data.size)


@pytest.mark.parametrize("n", [700, 5000, 10_000, 21_000])
def test_cbc_batched_many_messages(aes_lib_ready, orc, n):
    """aes_cbc_batched with enough messages (about half of them encrypted) to reach every
    four-lane shape on a 152-SM GB300 (one, several and eight chains per warp) and the one-lane
    kernel (21,000): AES-128/256 keys, both directions, lengths 0-6 blocks; sampled messages
    against the oracle's CBC, and every encrypted message decrypts back."""
    rng = np.random.default_rng(90 + n)
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8) for b in (128, 256, 128)]
    key_idx = rng.integers(0, len(keys), n).astype(np.uint32)
    dirs = rng.integers(0, 2, n).astype(np.uint32)
    lengths = (rng.integers(0, 7, n) * 16).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["dir"], msgs["offset"], msgs["length"] = key_idx, dirs, offsets, lengths
    with aes.KeyPool(len(keys)) as pool:
        for i, k in enumerate(keys):
            pool.load_keys(i, k[None, :], 8 * len(k))
        x = dev(data)
        y = x.clone()
        aes.aes_cbc_batched(pool, msgs, ivs, x.data_ptr(), y.data_ptr(), data.size)
        got = host(y)
        for i in np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 300)])):
            o, L = int(offsets[i]), int(lengths[i])
            if not L:
                continue
            f = orc.cbc_decrypt if dirs[i] else orc.cbc_encrypt
            assert np.array_equal(got[o:o + L], f(keys[int(key_idx[i])], ivs[i], data[o:o + L])), i
        back = msgs.copy()
        back["dir"] = 1
        back["length"] = np.where(dirs == 0, lengths, 0)
        z = y.clone()
        aes.aes_cbc_batched(pool, back, ivs, y.data_ptr(), z.data_ptr(), data.size)
        zz = host(z)
        for i in np.nonzero((dirs == 0) & (lengths > 0))[0]:
            o, L = int(offsets[i]), int(lengths[i])
            assert np.array_equal(zz[o:o + L], data[o:o + L]), i


def test_cbc_batched_encrypt_in_place(aes_lib_ready, orc):
    """aes_cbc_batched encryption with the output buffer the input buffer (allowed for
    encryption: each chain reads its next block before it overwrites the current one), 300
    messages of 1-40 blocks with own keys and IVs, every message against the oracle."""
    rng = np.random.default_rng(95)
    n = 300
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8) for b in (128, 192, 256)]
    key_idx = rng.integers(0, len(keys), n).astype(np.uint32)
    lengths = (rng.integers(1, 41, n) * 16).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["offset"], msgs["length"] = key_idx, offsets, lengths
    with aes.KeyPool(len(keys)) as pool:
        for i, k in enumerate(keys):
            pool.load_keys(i, k[None, :], 8 * len(k))
        x = dev(data)
        aes.aes_cbc_batched(pool, msgs, ivs, x.data_ptr(), x.data_ptr(), data.size)
        got = host(x)
        for i in range(n):
            o, L = int(offsets[i]), int(lengths[i])
            assert np.array_equal(got[o:o + L], orc.cbc_encrypt(keys[int(key_idx[i])], ivs[i], data[o:o + L])), i
