"""aes_crypt_batched_noalloc: the batched cipher for callers that may not allocate device
memory (a plug-in inside a host application that owns all device memory, or a path where
cudaMalloc's implicit device synchronisation is not acceptable).  It keeps its working data
in a fixed array the library declares in device memory, so the caller hands over only keys,
messages, input and output.

Checked through the C ABI against the pool-based entry point (aes_crypt_batched) on two
calls in a row, the second smaller than the first, so stale contents of the shared array
would show.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes
from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu


def _schedules(keys, bits):
    arr = (aes.aes_key_schedule * len(keys))()
    for i, k in enumerate(keys):
        arr[i] = aes.aes_key_expand(bytes(k), bits)
    return arr


def _noalloc(lib, scheds, nkeys, msgs, d_in, d_out, nbytes, stream):
    m = np.ascontiguousarray(msgs, dtype=aes.msg_dtype())
    return lib.aes_crypt_batched_noalloc(scheds, nkeys, m.ctypes.data, m.shape[0], d_in, d_out, nbytes, stream)


def test_noalloc_matches_pool_path_on_two_calls(aes_lib_ready):
    import torch

    lib = aes.lib()
    lib.aes_crypt_batched_noalloc.restype = ctypes.c_int
    lib.aes_crypt_batched_noalloc.argtypes = [ctypes.POINTER(aes.aes_key_schedule), ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_void_p]
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(60)
    # first call: 256 keys (128 AES-128, 128 AES-256), 4096 messages of both directions
    keys128 = rng.integers(0, 256, (128, 16), dtype=np.uint8)
    keys256 = rng.integers(0, 256, (128, 32), dtype=np.uint8)
    scheds = (aes.aes_key_schedule * 256)()
    for i in range(128):
        scheds[i] = aes.aes_key_expand(keys128[i].tobytes(), 128)
        scheds[128 + i] = aes.aes_key_expand(keys256[i].tobytes(), 256)
    m1 = workloads.batched_messages(61, m=4096, median=1024.0, hi=1 << 18)
    msgs1 = np.zeros(4096, dtype=aes.msg_dtype())
    msgs1["key_idx"] = rng.integers(0, 256, 4096)
    msgs1["dir"] = rng.integers(0, 2, 4096)
    msgs1["offset"], msgs1["length"] = m1.offsets, m1.lengths
    # second call: fewer keys and messages, encryption only, so leftovers of call 1 would show
    m2 = workloads.batched_messages(62, m=100, median=4096.0, hi=1 << 20)
    scheds2 = (aes.aes_key_schedule * 3)(*(aes.aes_key_expand(m2.keys[i].tobytes(), 128) for i in range(3)))
    msgs2 = np.zeros(100, dtype=aes.msg_dtype())
    msgs2["key_idx"] = np.arange(100) % 3
    msgs2["offset"], msgs2["length"] = m2.offsets, m2.lengths

    with aes.KeyPool(256) as pool:
        pool.load_keys(0, keys128, 128)
        pool.load_keys(128, keys256, 256)
        x1 = torch.from_numpy(m1.data).cuda()
        ref1 = torch.empty_like(x1)
        aes.aes_crypt_batched(pool, msgs1, x1.data_ptr(), ref1.data_ptr(), x1.numel())
        out1 = torch.empty_like(x1)
        assert _noalloc(lib, scheds, 256, msgs1, x1.data_ptr(), out1.data_ptr(), x1.numel(), stream) == aes.AES_OK

        x2 = torch.from_numpy(m2.data).cuda()
        out2 = torch.empty_like(x2)
        assert _noalloc(lib, scheds2, 3, msgs2, x2.data_ptr(), out2.data_ptr(), x2.numel(), stream) == aes.AES_OK
        with aes.KeyPool(3) as pool2:
            for i in range(3):
                pool2.set(i, scheds2[i])
            ref2 = torch.empty_like(x2)
            aes.aes_crypt_batched(pool2, msgs2, x2.data_ptr(), ref2.data_ptr(), x2.numel())
            torch.cuda.synchronize()
            assert torch.equal(out1, ref1)
            assert torch.equal(out2, ref2)


def test_noalloc_limits_and_errors(aes_lib_ready):
    import torch

    lib = aes.lib()
    lib.aes_crypt_batched_noalloc.restype = ctypes.c_int
    lib.aes_crypt_batched_noalloc.argtypes = [ctypes.POINTER(aes.aes_key_schedule), ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_void_p]
    x = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    scheds = (aes.aes_key_schedule * 257)(*(aes.aes_key_expand(bytes(16)) for _ in range(257)))
    ok = np.zeros(1, dtype=aes.msg_dtype())
    ok["length"] = 64
    assert _noalloc(lib, scheds, 257, ok, x.data_ptr(), x.data_ptr(), x.numel(), None) == aes.AES_EINVAL
    assert "static maximum" in aes.aes_last_error()
    many = np.zeros(4097, dtype=aes.msg_dtype())
    many["length"] = 16
    assert _noalloc(lib, scheds, 1, many, x.data_ptr(), x.data_ptr(), x.numel(), None) == aes.AES_EINVAL
    assert "static maximum" in aes.aes_last_error()
    bad = ok.copy()
    bad["key_idx"] = 5
    assert _noalloc(lib, scheds, 2, bad, x.data_ptr(), x.data_ptr(), x.numel(), None) == aes.AES_EINVAL
