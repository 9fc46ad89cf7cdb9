"""GPU parity of every compiled launch shape of the independent-block T-table kernel against
the CPU oracle, bit-exact.

The launch tuner may pick any (CTA threads, blocks in flight per thread) pair the library
compiles, and the benchmark times the pair it picks, so each pair is pinned here directly
(set as the AES_IMPL_AUTO choice, then called through aes_crypt_blocks): both directions,
AES-128/192/256 (10, 12 and 14 rounds, App. A1/A4 for the cipher, App. A3 and the AES
standard's word rule for the schedules), ragged sizes from one block to past one full wave of
the largest CTA shape, and an IV.  Decryption is checked on arbitrary data, not only on
ciphertext.  The last test compares the whole 1 GiB benchmark buffer (2^26 blocks, seed 1)
with the oracle for every shape and for the bitsliced kernel.
"""
import functools
import os

import numpy as np
import pytest

from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4

# every (threads, blocks per thread) pair compiled for the T-table kernel
SHAPES = [(256, 4), (512, 1), (512, 2), (512, 4), (768, 2), (1024, 1), (1024, 2)]
SHAPE_IDS = [f"{t}x{u}" for t, u in SHAPES]
# ragged sizes: a single block, partial warps and CTAs, the grid-stride loop's tail, and one
# size past a full wave of 768-thread CTAs x 2 blocks on 152 SMs (233,472 blocks)
SIZES = [1, 33, 1025, 77_825, 155_651, 237_571]


@pytest.fixture
def shape(request, aes_lib_ready):
    """Pins the AES_IMPL_AUTO choice to one T-table shape for every direction and round count
    (so that small calls take it too), and clears it afterwards."""
    aes = aes_lib_ready
    t, u = request.param

    def put(impl, tt, uu):
        for d in ("encrypt", "decrypt"):
            for nr in (10, 12, 14):
                aes.aes_set_auto_choice(d, nr, impl, tt, uu)

    put("ttable", t, u)
    yield t, u
    put("auto", 0, 0)


@functools.lru_cache(maxsize=None)
def _case(key_bits: int, n: int, with_iv: bool):
    rng = np.random.default_rng(1000 * key_bits + n + (7 if with_iv else 0))
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    iv = rng.integers(0, 256, 16, dtype=np.uint8) if with_iv else None
    data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
    return key, iv, data


@functools.lru_cache(maxsize=None)
def _want(orc, key_bits: int, n: int, with_iv: bool, decrypt: bool):
    key, iv, data = _case(key_bits, n, with_iv)
    fn = orc.decrypt_blocks if decrypt else orc.encrypt_blocks
    return fn(key, data, iv=iv, threads=THREADS)


def _run(aes, key, iv, data, direction):
    import torch

    ks = aes.aes_key_expand(key.tobytes(), 8 * len(key))
    x = torch.from_numpy(data).cuda()
    y = aes.crypt(x, ks, direction, iv=None if iv is None else iv.tobytes(), impl="auto")
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS, indirect=True)
@pytest.mark.parametrize("key_bits", [128, 192, 256])
@pytest.mark.parametrize("n", SIZES)
def test_shape_against_oracle(aes_lib_ready, orc, shape, key_bits, n):
    aes = aes_lib_ready
    key, iv, data = _case(key_bits, n, False)
    assert (_run(aes, key, iv, data, "encrypt") == _want(orc, key_bits, n, False, False)).all()
    assert (_run(aes, key, iv, data, "decrypt") == _want(orc, key_bits, n, False, True)).all()


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS, indirect=True)
@pytest.mark.parametrize("key_bits", [128, 256])
def test_shape_with_iv(aes_lib_ready, orc, shape, key_bits):
    aes = aes_lib_ready
    n = 155_651
    key, iv, data = _case(key_bits, n, True)
    assert (_run(aes, key, iv, data, "encrypt") == _want(orc, key_bits, n, True, False)).all()
    assert (_run(aes, key, iv, data, "decrypt") == _want(orc, key_bits, n, True, True)).all()


@pytest.fixture(scope="module")
def gib(orc):
    """The benchmark's buffer (2^26 blocks of seed-1 data, its AES-128 key) and the oracle's
    whole ciphertext of it (about 20 s on 16 cores)."""
    w = workloads.plain(1, 1 << 26)
    return w, orc.encrypt_blocks(w.key, w.data, threads=THREADS)


@pytest.mark.parametrize("impl", [f"ttable-{s}" for s in SHAPE_IDS] + ["bitslice"])
def test_whole_1gib_buffer(aes_lib_ready, gib, impl):
    """Every byte of the 1 GiB encryption equals the oracle's, at each launch shape (the one the
    launch tuner picks for the benchmark among them); decryption restores every byte."""
    import torch

    aes = aes_lib_ready
    w, want = gib
    ks = aes.aes_key_expand(w.key.tobytes())
    if impl.startswith("ttable-"):
        t, u = (int(v) for v in impl[len("ttable-"):].split("x"))
        for d in ("encrypt", "decrypt"):
            aes.aes_set_auto_choice(d, 10, "ttable", t, u)
        which = "auto"
    else:
        which = "bitslice"
    try:
        x = torch.from_numpy(w.data).cuda()
        ct = aes.encrypt(x, ks, impl=which)
        torch.cuda.synchronize()
        assert np.array_equal(ct.cpu().numpy(), want)
        pt = aes.decrypt(ct, ks, impl=which)
        torch.cuda.synchronize()
        assert torch.equal(pt, x)
        del x, ct, pt
        torch.cuda.empty_cache()
    finally:
        for d in ("encrypt", "decrypt"):
            aes.aes_set_auto_choice(d, 10, "auto", 0, 0)
