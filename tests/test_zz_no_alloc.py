"""aes_crypt_batched_noalloc: the batched cipher for callers that may not allocate device
memory (a plug-in inside a host application that owns all device memory, or a path where
cudaMalloc's implicit device synchronisation is not acceptable).  It keeps its working data
in a fixed array the library declares in device memory, so the caller hands over only keys,
messages, input and output.

Checked through the C ABI against the CPU oracle, message by message, on two calls in a
row, the second smaller than the first, so stale contents of the shared array would show;
the output also equals the pool-based entry point's (aes_crypt_batched).  A second call
must leave the device's free memory unchanged, and a capturing stream is refused.  This
file is collected last on purpose.
"""
import ctypes
import os

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes
from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


def _declare(lib):
    lib.aes_crypt_batched_noalloc.restype = ctypes.c_int
    lib.aes_crypt_batched_noalloc.argtypes = [ctypes.POINTER(aes.aes_key_schedule), ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_void_p]
    return lib


def _noalloc(lib, scheds, nkeys, msgs, d_in, d_out, nbytes, stream):
    m = np.ascontiguousarray(msgs, dtype=aes.msg_dtype())
    return lib.aes_crypt_batched_noalloc(scheds, nkeys, m.ctypes.data, m.shape[0], d_in, d_out, nbytes, stream)


def _oracle_out(orc, keys, msgs, data: np.ndarray) -> np.ndarray:
    """The expected output buffer: every message under its own key and direction (one oracle
    call per (key, direction) group of messages); bytes outside the messages are unchanged
    from `data`, which the callers also place in the output buffer beforehand."""
    out = data.copy()
    groups = {}
    for i in range(len(msgs)):
        if msgs["length"][i]:
            groups.setdefault((int(msgs["key_idx"][i]), int(msgs["dir"][i])), []).append(i)
    for (k, d), idx in groups.items():
        src = np.concatenate([data[int(msgs["offset"][i]):int(msgs["offset"][i] + msgs["length"][i])] for i in idx])
        got = (orc.decrypt_blocks if d else orc.encrypt_blocks)(keys[k], src, threads=THREADS)
        pos = 0
        for i in idx:
            o, L = int(msgs["offset"][i]), int(msgs["length"][i])
            out[o:o + L] = got[pos:pos + L]
            pos += L
    return out


def test_noalloc_matches_oracle_on_two_calls(aes_lib_ready, orc):
    import torch

    lib = _declare(aes.lib())
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(60)
    # first call: 256 keys (128 AES-128, 128 AES-256), 4096 messages of both directions
    keys = [rng.integers(0, 256, 16, dtype=np.uint8) for _ in range(128)] + \
           [rng.integers(0, 256, 32, dtype=np.uint8) for _ in range(128)]
    scheds = (aes.aes_key_schedule * 256)(*(aes.aes_key_expand(k.tobytes(), 8 * len(k)) for k in keys))
    m1 = workloads.batched_messages(61, m=4096, median=1024.0, hi=1 << 18)
    msgs1 = np.zeros(4096, dtype=aes.msg_dtype())
    msgs1["key_idx"] = rng.integers(0, 256, 4096)
    msgs1["dir"] = rng.integers(0, 2, 4096)
    msgs1["offset"], msgs1["length"] = m1.offsets, m1.lengths
    msgs1["length"][::97] = 0  # empty messages are skipped
    # second call: fewer keys and messages, encryption only, so leftovers of call 1 would show
    m2 = workloads.batched_messages(62, m=100, median=4096.0, hi=1 << 20)
    keys2 = [m2.keys[i] for i in range(3)]
    scheds2 = (aes.aes_key_schedule * 3)(*(aes.aes_key_expand(k.tobytes(), 128) for k in keys2))
    msgs2 = np.zeros(100, dtype=aes.msg_dtype())
    msgs2["key_idx"] = np.arange(100) % 3
    msgs2["offset"], msgs2["length"] = m2.offsets, m2.lengths

    x1 = torch.from_numpy(m1.data).cuda()
    out1 = x1.clone()
    assert _noalloc(lib, scheds, 256, msgs1, x1.data_ptr(), out1.data_ptr(), x1.numel(), stream) == aes.AES_OK
    torch.cuda.synchronize()
    x2 = torch.from_numpy(m2.data).cuda()
    out2 = x2.clone()
    free_before, _ = torch.cuda.mem_get_info()
    assert _noalloc(lib, scheds2, 3, msgs2, x2.data_ptr(), out2.data_ptr(), x2.numel(), stream) == aes.AES_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, "the second call changed the device's free memory"

    assert (out1.cpu().numpy() == _oracle_out(orc, keys, msgs1, m1.data)).all()
    assert (out2.cpu().numpy() == _oracle_out(orc, keys2, msgs2, m2.data)).all()

    # the same output as the pool-based entry point
    with aes.KeyPool(256) as pool:
        for i in range(256):
            pool.set(i, scheds[i])
        ref1 = x1.clone()
        aes.aes_crypt_batched(pool, msgs1, x1.data_ptr(), ref1.data_ptr(), x1.numel())
        torch.cuda.synchronize()
        assert torch.equal(out1, ref1)


def test_noalloc_refuses_a_capturing_stream(aes_lib_ready):
    import torch

    lib = _declare(aes.lib())
    x = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    y = torch.zeros_like(x)
    scheds = (aes.aes_key_schedule * 1)(aes.aes_key_expand(bytes(16)))
    msgs = np.zeros(1, dtype=aes.msg_dtype())
    msgs["length"] = x.numel()
    # a call outside capture first: the device set-up is done before any capture
    assert _noalloc(lib, scheds, 1, msgs, x.data_ptr(), y.data_ptr(), x.numel(),
                    torch.cuda.current_stream().cuda_stream) == aes.AES_OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    rc = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            y.add_(0)  # the graph holds one node of torch's own
            rc = _noalloc(lib, scheds, 1, msgs, x.data_ptr(), y.data_ptr(), x.numel(), s.cuda_stream)
        finally:
            g.capture_end()
    assert rc == aes.AES_EINVAL
    assert "captured" in aes.aes_last_error()
    del g


def test_noalloc_limits_and_errors(aes_lib_ready):
    import torch

    lib = _declare(aes.lib())
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
