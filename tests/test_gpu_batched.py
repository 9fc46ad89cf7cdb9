"""GPU parity of the key pool and the batched persistent launch, through the C ABI.

References: the CPU oracle (per message, its own key) and the single-key kernel path
(already pinned to the oracle) for the full 4096-message lognormal workload.  All
comparisons are bit-exact.
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


def msgs_for(m: workloads.Messages, dirs=None, key_idx=None):
    out = np.zeros(len(m.lengths), dtype=aes.msg_dtype())
    out["key_idx"] = np.arange(len(m.lengths)) if key_idx is None else key_idx
    out["dir"] = 0 if dirs is None else dirs
    out["offset"] = m.offsets
    out["length"] = m.lengths
    return out


def test_batched_4096_lognormal_messages(aes_lib_ready, orc):
    import torch

    m = workloads.batched_messages(3)
    total = int(m.lengths.sum())
    with aes.KeyPool(len(m.keys)) as pool:
        pool.load_keys(0, m.keys, 128)
        assert pool.rounds(0) == 10 and pool.rounds(4095) == 10
        x = dev(m.data)
        y = torch.empty_like(x)
        msgs = msgs_for(m)
        aes.aes_crypt_batched(pool, msgs, x.data_ptr(), y.data_ptr(), total)
        got = host(y)
        # oracle on a spread of whole messages (short and long ones)
        rng = np.random.default_rng(30)
        pick = np.unique(np.concatenate([rng.integers(0, len(m.keys), 48), [int(np.argmax(m.lengths)), 0, 4095]]))
        for i in pick:
            o, L = int(m.offsets[i]), int(m.lengths[i])
            if L > 16 * 40_000:  # long messages: sample 4096 blocks, the oracle is slow
                idx = np.unique(rng.integers(0, L // 16, 4096))
                src = m.data[o:o + L].reshape(-1, 16)[idx].reshape(-1)
                want = orc.encrypt_blocks(m.keys[i], src, threads=THREADS)
                assert (got[o:o + L].reshape(-1, 16)[idx].reshape(-1) == want).all(), i
            else:
                assert (got[o:o + L] == orc.encrypt_blocks(m.keys[i], m.data[o:o + L], threads=THREADS)).all(), i
        # every message against the single-key kernel with a host-expanded schedule
        ref = torch.empty_like(x)
        for i in range(len(m.keys)):
            o, L = int(m.offsets[i]), int(m.lengths[i])
            ks = aes.aes_key_expand(m.keys[i].tobytes())
            aes.aes_crypt_blocks(ks, None, x.data_ptr() + o, ref.data_ptr() + o, L // 16, "encrypt", "ttable")
        torch.cuda.synchronize()
        assert torch.equal(ref, y)
        # decrypting the batch restores the plaintext
        msgs["dir"] = 1
        z = torch.empty_like(x)
        aes.aes_crypt_batched(pool, msgs, y.data_ptr(), z.data_ptr(), total)
        torch.cuda.synchronize()
        assert torch.equal(z, x)


def test_every_shape_gives_identical_output(aes_lib_ready):
    import torch

    m = workloads.batched_messages(31, m=300, median=2048.0, hi=1 << 20)
    total = int(m.lengths.sum())
    with aes.KeyPool(len(m.keys)) as pool:
        pool.load_keys(0, m.keys, 128)
        x = dev(m.data)
        msgs = msgs_for(m)
        outs = []
        with aes.Batch(pool, 512) as b:
            for shape in [(512, 1), (512, 2), (512, 4), (384, 4), (256, 4), (768, 1)]:
                b.set_shape(*shape)
                y = torch.empty_like(x)
                b.run(msgs, x.data_ptr(), y.data_ptr(), total)
                b.run(msgs, x.data_ptr(), y.data_ptr(), total)  # second run replays the cached graph
                torch.cuda.synchronize()
                outs.append(y)
            with pytest.raises(aes.AesError):
                b.set_shape(384, 3)
        for o in outs[1:]:
            assert torch.equal(o, outs[0])


@pytest.mark.parametrize("case", ["enc128-decmixed", "encmixed-dec128", "both128", "dec128-only", "mixed"])
def test_round_specialised_kernels(aes_lib_ready, orc, case):
    """A direction whose messages all use AES-128 keys runs a body specialised to 10 rounds (and
    the 768-thread shape exists only for AES-128 throughout; other work set to that shape runs
    the generic 512-thread kernel).  Every combination of specialised and generic directions,
    with AES-128, -192 and -256 keys, at every shape that has specialisations, matches the
    oracle."""
    import torch

    rng = np.random.default_rng(40 + len(case))
    n = 120
    third = n // 3
    keys = [rng.integers(0, 256, (third, b // 8), dtype=np.uint8) for b in (128, 192, 256)]
    lengths = (rng.integers(1, 200, n) * 16).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    dirs = rng.integers(0, 2, n).astype(np.uint32)
    if case == "dec128-only":
        dirs[:] = 1
    small = rng.integers(0, third, n)            # AES-128 slots
    any_ = rng.integers(0, n, n)                 # any size
    enc128 = case in ("enc128-decmixed", "both128")
    dec128 = case in ("encmixed-dec128", "both128", "dec128-only")
    key_idx = np.where(dirs == 0, np.where(enc128, small, any_), np.where(dec128, small, any_)).astype(np.uint32)
    with aes.KeyPool(n) as pool:
        for j, bits in enumerate((128, 192, 256)):
            pool.load_keys(j * third, keys[j], bits)
        msgs = np.zeros(n, dtype=aes.msg_dtype())
        msgs["key_idx"], msgs["dir"], msgs["offset"], msgs["length"] = key_idx, dirs, offsets, lengths
        x = dev(data)
        with aes.Batch(pool, n) as b:
            for shape in [(512, 1), (512, 2), (768, 1)]:
                b.set_shape(*shape)
                y = torch.empty_like(x)
                b.run(msgs, x.data_ptr(), y.data_ptr(), data.size)
                got = host(y)
                for i in range(n):
                    o, L = int(offsets[i]), int(lengths[i])
                    k = int(key_idx[i])
                    key = keys[k // third][k % third]
                    f = orc.encrypt_blocks if dirs[i] == 0 else orc.decrypt_blocks
                    assert (got[o:o + L] == f(key, data[o:o + L], threads=THREADS)).all(), (shape, i)


def test_mixed_directions_key_sizes_empty_and_in_place(aes_lib_ready, orc):
    import torch

    rng = np.random.default_rng(32)
    n = 200
    keys128 = rng.integers(0, 256, (n // 2, 16), dtype=np.uint8)
    keys256 = rng.integers(0, 256, (n // 2, 32), dtype=np.uint8)
    lengths = (rng.integers(0, 300, n) * 16).astype(np.int64)
    lengths[::17] = 0  # empty messages are allowed
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    dirs = rng.integers(0, 2, n).astype(np.uint32)
    key_idx = rng.permutation(n).astype(np.uint32)  # slots 0..99 AES-128, 100..199 AES-256
    with aes.KeyPool(n) as pool:
        pool.load_keys(0, keys128, 128)
        pool.load_keys(n // 2, keys256, 256)
        assert pool.rounds(0) == 10 and pool.rounds(n - 1) == 14
        msgs = np.zeros(n, dtype=aes.msg_dtype())
        msgs["key_idx"], msgs["dir"], msgs["offset"], msgs["length"] = key_idx, dirs, offsets, lengths
        x = dev(data)
        aes.aes_crypt_batched(pool, msgs, x.data_ptr(), x.data_ptr(), data.size)  # in place
        got = host(x)
        for i in range(n):
            o, L = int(offsets[i]), int(lengths[i])
            k = int(key_idx[i])
            key = keys128[k] if k < n // 2 else keys256[k - n // 2]
            f = orc.encrypt_blocks if dirs[i] == 0 else orc.decrypt_blocks
            want = f(key, data[o:o + L], threads=THREADS) if L else data[o:o + L]
            assert (got[o:o + L] == want).all(), i


def test_pool_set_matches_device_expansion(aes_lib_ready):
    import torch

    rng = np.random.default_rng(33)
    for bits in (128, 192, 256):
        keys = rng.integers(0, 256, (64, bits // 8), dtype=np.uint8)
        data = rng.integers(0, 256, 64 * 16 * 37, dtype=np.uint8)
        msgs = np.zeros(128, dtype=aes.msg_dtype())
        for j in range(128):
            msgs[j] = (j % 64, j // 64, (j % 64) * 16 * 37, 16 * 37)
        msgs = msgs[np.argsort(msgs["dir"], kind="stable")]
        # first 64 messages encrypt, the next 64 decrypt (of the same regions, out of place)
        outs = []
        for use_device in (True, False):
            with aes.KeyPool(64) as pool:
                if use_device:
                    pool.load_keys(0, keys, bits)
                else:
                    for i in range(64):
                        pool.set(i, aes.aes_key_expand(keys[i].tobytes(), bits))
                x = dev(data)
                y = torch.empty_like(x)
                aes.aes_crypt_batched(pool, msgs[:64], x.data_ptr(), y.data_ptr(), data.size)
                z = torch.empty_like(x)
                aes.aes_crypt_batched(pool, msgs[64:], y.data_ptr(), z.data_ptr(), data.size)
                torch.cuda.synchronize()
                assert torch.equal(z, x)
                outs.append(y)
        assert torch.equal(outs[0], outs[1])


def test_autotune_and_cache(aes_lib_ready, tmp_path):
    import json

    import torch

    m = workloads.batched_messages(34, m=512)
    total = int(m.lengths.sum())
    cache = tmp_path / "tune.json"
    with aes.KeyPool(len(m.keys)) as pool:
        pool.load_keys(0, m.keys, 128)
        x = dev(m.data)
        y = torch.empty_like(x)
        msgs = msgs_for(m)
        with aes.Batch(pool, 1024) as b:
            shape = b.autotune(msgs, x.data_ptr(), y.data_ptr(), total, str(cache))
            assert shape in [(512, 1), (512, 2), (512, 4), (384, 4), (256, 4), (768, 1)]
            entries = json.loads(cache.read_text())
            assert len(entries) == 1
            (sig, val), = entries.items()
            assert (val["threads"], val["blocks_per_lane"]) == shape and val["us"] > 0
            # a second tune on the same workload reuses the cache entry
            assert b.autotune(msgs, x.data_ptr(), y.data_ptr(), total, str(cache)) == shape
            b.run(msgs, x.data_ptr(), y.data_ptr(), total)
            ref = torch.empty_like(x)
            aes.aes_crypt_batched(pool, msgs, x.data_ptr(), ref.data_ptr(), total)
            torch.cuda.synchronize()
            assert torch.equal(ref, y)


def test_batched_argument_errors(aes_lib_ready):
    import torch

    with aes.KeyPool(4) as pool:
        pool.load_keys(0, np.zeros((2, 16), dtype=np.uint8), 128)
        x = torch.zeros(4096, dtype=torch.uint8, device="cuda")
        y = torch.zeros_like(x)
        bad = [
            [(2, 0, 0, 64)],        # slot 2 never loaded
            [(9, 0, 0, 64)],        # slot beyond capacity
            [(0, 0, 8, 64)],        # offset not a multiple of 16
            [(0, 0, 0, 24)],        # length not a multiple of 16
            [(0, 0, 4080, 32)],     # leaves the buffer
            [(0, 3, 0, 64)],        # bad direction
        ]
        for msgs in bad:
            with pytest.raises(aes.AesError) as ei:
                aes.aes_crypt_batched(pool, msgs, x.data_ptr(), y.data_ptr(), 4096)
            assert ei.value.status == aes.AES_EINVAL
        with pytest.raises(aes.AesError):
            pool.load_keys(3, np.zeros((2, 16), dtype=np.uint8), 128)  # slots 3..4 > capacity
        with pytest.raises(aes.AesError):
            aes.aes_crypt_batched(pool, [(0, 0, 0, 64)], x.data_ptr(), x.data_ptr() + 16, 4096)  # overlap
