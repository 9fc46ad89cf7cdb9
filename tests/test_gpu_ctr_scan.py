"""GPU parity of counter mode (against the oracle's CTR, itself pinned to OpenSSL) and of the
equality scan over an encrypted sensor column (against numpy record equality).  Bit-exact."""
import os

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes
from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.mark.parametrize("key_bits", [128, 192, 256])
@pytest.mark.parametrize("n", [1, 33, 100_003])
def test_ctr_matches_oracle(aes_lib_ready, orc, key_bits, n):
    import torch

    rng = np.random.default_rng(100 + n + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    ctr0 = rng.integers(0, 256, 16, dtype=np.uint8)
    ctr0[8:] = 0xFF  # the low 64 bits carry into the high half within the first blocks
    ctr0[15] = 0xF0
    data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    x = torch.from_numpy(data).cuda()
    ct = aes.ctr(x, ks, ctr0.tobytes()).cpu().numpy()
    assert (ct == orc.ctr_crypt(key, ctr0, data)).all()
    back = aes.ctr(torch.from_numpy(ct).cuda(), ks, ctr0.tobytes()).cpu().numpy()
    assert (back == data).all()


def test_ctr_full_wrap(aes_lib_ready, orc):
    import torch

    key = np.arange(16, dtype=np.uint8)
    ctr0 = np.full(16, 0xFF, dtype=np.uint8)  # wraps to zero after the first block
    data = np.zeros(16 * 4, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes())
    got = aes.ctr(torch.from_numpy(data).cuda(), ks, ctr0.tobytes()).cpu().numpy()
    assert (got == orc.ctr_crypt(key, ctr0, data)).all()


def test_equality_scan_on_encrypted_sensor_column(aes_lib_ready, orc):
    import torch

    col = workloads.sensor_records(2, 1_000_000)
    rec = col.records.reshape(-1, 16).copy()
    # plant repeats of three records so that the queries have several answers
    rng = np.random.default_rng(5)
    for src in (7, 123_456, 999_999):
        for dst in rng.integers(0, len(rec), 5):
            rec[dst] = rec[src]
    ks = aes.aes_key_expand(col.key128.tobytes())
    enc = aes.encrypt(torch.from_numpy(rec.reshape(-1)).cuda(), ks)
    for src in (7, 123_456, 999_999, 42):
        query = rec[src]
        needle = orc.encrypt_blocks(col.key128, query).tobytes()  # the client encrypts its query
        idx, k = aes.find_equal(enc, needle)
        want = np.flatnonzero((rec == query).all(axis=1))
        assert k == len(want)
        assert (idx.cpu().numpy() == want).all()
    # an absent value finds nothing; a small max_matches still counts every match
    idx, k = aes.find_equal(enc, bytes(16))
    assert k == 0 and idx.numel() == 0
    needle = orc.encrypt_blocks(col.key128, rec[7]).tobytes()
    idx, k = aes.find_equal(enc, needle, max_matches=2)
    assert k >= 2 and idx.numel() == 2


@pytest.mark.parametrize("n", [1, 5, 33, 311_297, 1_000_003])
def test_equality_scan_ragged_sizes(aes_lib_ready, n):
    """Record counts that end inside a warp, inside the first loads of a thread and past one
    grid-wide step of four loads per thread; matches planted at the first and last records and
    in between, checked against numpy record equality."""
    import torch

    rng = np.random.default_rng(6 + n)
    rec = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    needle = rng.integers(0, 256, 16, dtype=np.uint8)
    for dst in {0, n - 1, n // 2, n // 3}:
        rec[dst] = needle
    col = torch.from_numpy(rec.reshape(-1)).cuda()
    idx, k = aes.find_equal(col, needle.tobytes())
    want = np.flatnonzero((rec == needle).all(axis=1))
    assert k == len(want)
    assert (idx.cpu().numpy() == want).all()
