"""aes_crypt_host (host buffers) through the C ABI: pinned and pageable inputs, several 64 MiB
chunks with a ragged last one, in place, and an input that is not 16-byte aligned.  Compared
bit-exactly with the device-buffer entry point and, on sampled blocks, with the oracle."""
import os

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes
from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
N = 9_000_003  # 3 chunks of 4M blocks, the last one ragged


def device_reference(ks, data, d):
    import torch

    x = torch.from_numpy(data).cuda()
    return aes.crypt(x, ks, d).cpu().numpy()


@pytest.fixture(scope="module")
def work():
    w = workloads.plain(90, N)
    ks = aes.aes_key_expand(w.key.tobytes())
    return w, ks, device_reference(ks, w.data, "encrypt")


def test_pinned_buffers(aes_lib_ready, orc, work):
    import torch

    w, ks, ref = work
    hx = torch.from_numpy(w.data).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    aes.aes_crypt_host(ks, None, hx.data_ptr(), hy.data_ptr(), N, "encrypt")
    got = hy.numpy()
    assert (got == ref).all()
    idx = np.unique(np.random.default_rng(91).integers(0, N, 2000))
    want = orc.encrypt_blocks(w.key, w.data.reshape(-1, 16)[idx].reshape(-1), threads=THREADS)
    assert (got.reshape(-1, 16)[idx].reshape(-1) == want).all()
    # decrypt back, in place, from pinned memory
    aes.aes_crypt_host(ks, None, hy.data_ptr(), hy.data_ptr(), N, "decrypt")
    assert (hy.numpy() == w.data).all()


def test_pageable_buffers(aes_lib_ready, work):
    w, ks, ref = work
    out = np.empty_like(w.data)
    aes.aes_crypt_host(ks, None, w.data.ctypes.data, out.ctypes.data, N, "encrypt")
    assert (out == ref).all()
    buf = out.copy()
    aes.aes_crypt_host(ks, None, buf.ctypes.data, buf.ctypes.data, N, "decrypt")  # in place
    assert (buf == w.data).all()


def test_unaligned_pinned_input(aes_lib_ready, work):
    import torch

    w, ks, _ = work
    n = 300_001
    data = w.data[: 16 * n]
    hx = torch.empty(16 * n + 8, dtype=torch.uint8).pin_memory()
    hx[8:].copy_(torch.from_numpy(data))
    hy = torch.empty(16 * n, dtype=torch.uint8).pin_memory()
    iv = bytes(range(16))
    aes.aes_crypt_host(ks, iv, hx.data_ptr() + 8, hy.data_ptr(), n, "encrypt")
    import paper_1506_08503_gb300 as a

    x = torch.from_numpy(data.copy()).cuda()
    assert (hy.numpy() == a.crypt(x, ks, "encrypt", iv=iv).cpu().numpy()).all()
