"""Python binding of libaesgb.so: argument marshalling only.

Every function here forwards to the C ABI declared in include/aesgb.h with the same name;
all cipher work runs in the library's CUDA kernels.  PyTorch is used only to hand device
memory and streams to the library.  If the library is missing the import still works, but
every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libaesgb.so"

AES_OK = 0
AES_EINVAL = -1
AES_ENOMEM = -2
AES_ECUDA = -3
AES_EAGAIN = -4
AES_ETIMEDOUT = -5
AES_ENOTFOUND = -6

AES_ENCRYPT = 0
AES_DECRYPT = 1

AES_IMPL_AUTO = 0
AES_IMPL_TTABLE = 1
AES_IMPL_BITSLICE = 2

_IMPLS = {"auto": AES_IMPL_AUTO, "ttable": AES_IMPL_TTABLE, "bitslice": AES_IMPL_BITSLICE}
_DIRS = {"encrypt": AES_ENCRYPT, "decrypt": AES_DECRYPT, AES_ENCRYPT: AES_ENCRYPT, AES_DECRYPT: AES_DECRYPT}


class AesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"aesgb status {status}: {msg}")
        self.status = status


class aes_key_schedule(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("rk", (ctypes.c_uint8 * 16) * 15)]

    def round_keys(self) -> bytes:
        return bytes(bytearray(self.rk))[: 16 * (self.nr + 1)]


class aes_msg(ctypes.Structure):
    _fields_ = [("key_idx", ctypes.c_uint32), ("dir", ctypes.c_uint32), ("offset", ctypes.c_uint64),
                ("length", ctypes.c_uint64)]


_MSG_DTYPE = None


# numpy view of an aes_msg array (same layout, 24 bytes)
def msg_dtype():
    global _MSG_DTYPE
    if _MSG_DTYPE is None:
        import numpy as np
        _MSG_DTYPE = np.dtype([("key_idx", "<u4"), ("dir", "<u4"), ("offset", "<u8"), ("length", "<u8")])
    return _MSG_DTYPE


class aes_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("nstreams", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("queue_capacity", ctypes.c_uint32), ("fail_every", ctypes.c_uint32),
                ("linger_us", ctypes.c_uint32)]


class aes_request(ctypes.Structure):
    _fields_ = [("key_idx", ctypes.c_uint32), ("dir", ctypes.c_uint32), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("length", ctypes.c_uint64), ("src_on_device", ctypes.c_uint32),
                ("dst_on_device", ctypes.c_uint32)]


class aes_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "queued", "inflight", "launches",
                                                "bytes_completed")] + \
               [(n, ctypes.c_double) for n in ("p50_us", "p99_us", "max_us", "mean_us", "gbps", "mean_batch",
                                                "gbps_from_first_launch")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


AES_REQ_PENDING, AES_REQ_DONE, AES_REQ_FAILED = 0, 1, 2


def request_dtype():
    """numpy view of aes_request (40 bytes)."""
    import numpy as np
    return np.dtype([("key_idx", "<u4"), ("dir", "<u4"), ("src", "<u8"), ("dst", "<u8"), ("length", "<u8"),
                     ("src_on_device", "<u4"), ("dst_on_device", "<u4")])

_lib = None

# name -> (restype, argtypes)
_VP, _SZ, _I, _U8P = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)
_KSP = ctypes.POINTER(aes_key_schedule)
_SIGS: dict[str, tuple] = {
    "aes_last_error": (ctypes.c_char_p, []),
    "aes_version": (ctypes.c_char_p, []),
    "aes_key_expand": (_I, [_U8P, _I, _KSP]),
    "aes_encrypt_blocks": (_I, [_KSP, _U8P, _VP, _VP, _SZ, _VP]),
    "aes_decrypt_blocks": (_I, [_KSP, _U8P, _VP, _VP, _SZ, _VP]),
    "aes_crypt_blocks": (_I, [_KSP, _U8P, _VP, _VP, _SZ, _I, _I, _VP]),
    "aes_crypt_host": (_I, [_KSP, _U8P, _VP, _VP, _SZ, _I, _I, _VP]),
    "aes_cbc_crypt": (_I, [_KSP, _VP, _I, _VP, _VP, _SZ, _SZ, _I, _VP]),
    "aes_ctr_crypt": (_I, [_KSP, _U8P, _VP, _VP, _SZ, _VP]),
    "aes_scan_equal": (_I, [_VP, _SZ, _U8P, _VP, _SZ, _VP, _VP]),
    "aes_autotune_blocks": (_I, [_KSP, _VP, _VP, _SZ, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I), _VP]),
    "aes_set_auto_choice": (_I, [_I, _I, _I, _I, _I]),
    "aes_gcm_workspace_bytes": (_SZ, []),
    "aes_gcm_crypt": (_I, [_KSP, _U8P, _SZ, _VP, _SZ, _VP, _VP, _SZ, _I, _VP, _VP, _SZ, _VP]),
    "aes_gcm_decrypt_verify": (_I, [_KSP, _U8P, _SZ, _VP, _SZ, _VP, _VP, _SZ, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "aes_crypt_batched_noalloc": (_I, [_KSP, ctypes.c_uint32, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_keypool_create": (_I, [_SZ, ctypes.POINTER(_VP)]),
    "aes_keypool_load_keys": (_I, [_VP, ctypes.c_uint32, _SZ, _U8P, _I, _VP]),
    "aes_keypool_set": (_I, [_VP, ctypes.c_uint32, _KSP]),
    "aes_keypool_rounds": (_I, [_VP, ctypes.c_uint32]),
    "aes_keypool_destroy": (_I, [_VP]),
    "aes_batch_create": (_I, [_VP, _SZ, ctypes.POINTER(_VP)]),
    "aes_batch_run": (_I, [_VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_batch_autotune": (_I, [_VP, _VP, _SZ, _VP, _VP, _SZ, ctypes.c_char_p, ctypes.POINTER(_I),
                                ctypes.POINTER(_I), _VP]),
    "aes_batch_run_iv": (_I, [_VP, _VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_batch_set_shape": (_I, [_VP, _I, _I]),
    "aes_batch_destroy": (_I, [_VP]),
    "aes_crypt_batched": (_I, [_VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_crypt_batched_iv": (_I, [_VP, _VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_cbc_batched": (_I, [_VP, _VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "aes_server_create": (_I, [ctypes.POINTER(aes_server_cfg), _VP, ctypes.POINTER(_VP)]),
    "aes_server_submit": (_I, [_VP, ctypes.POINTER(aes_request), ctypes.POINTER(ctypes.c_uint64)]),
    "aes_server_submit_many": (_I, [_VP, _VP, _SZ, _VP]),
    "aes_server_poll": (_I, [_VP, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(_I)]),
    "aes_server_stats": (_I, [_VP, ctypes.POINTER(aes_stats)]),
    "aes_server_stats_get": (_I, [_VP, ctypes.POINTER(aes_stats)]),
    "aes_server_stats_reset": (_I, [_VP]),
    "aes_server_destroy": (_I, [_VP]),
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built (run build() first)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1506_08503_gb300.build()")
        l = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in _SIGS.items():
            f = getattr(l, name)
            f.restype, f.argtypes = res, args
        _lib = l
    return _lib


def _dir(d) -> int:
    """Direction name or number; unknown numbers pass through so the library rejects them."""
    return _DIRS[d] if isinstance(d, str) else int(d)


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _check(st: int) -> int:
    if st != AES_OK:
        raise AesError(st, (lib().aes_last_error() or b"").decode())
    return st


def _bytes_ptr(b):
    if b is None:
        return None
    buf = (ctypes.c_uint8 * len(b)).from_buffer_copy(bytes(b))
    return ctypes.cast(buf, _U8P), buf


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # no torch / no CUDA: legacy default stream
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- raw C-ABI mirrors ---------------------------------------------------------------------

def aes_last_error() -> str:
    return (lib().aes_last_error() or b"").decode()


def aes_version() -> str:
    return lib().aes_version().decode()


def aes_key_expand(key: bytes, key_bits: int | None = None) -> aes_key_schedule:
    key = bytes(key)
    key_bits = key_bits or 8 * len(key)
    if len(key) * 8 != key_bits:
        raise ValueError("key length does not match key_bits")
    ks = aes_key_schedule()
    p, _keep = _bytes_ptr(key)
    _check(lib().aes_key_expand(p, key_bits, ctypes.byref(ks)))
    return ks


def aes_crypt_blocks(ks: aes_key_schedule, iv, d_in: int, d_out: int, nblocks: int, dir, impl="auto",
                     stream=None) -> None:
    ivp = _bytes_ptr(iv)
    _check(lib().aes_crypt_blocks(ctypes.byref(ks), ivp[0] if ivp else None, d_in, d_out, nblocks,
                                  _dir(dir), _IMPLS[impl] if isinstance(impl, str) else int(impl),
                                  _stream_ptr(stream)))


def aes_encrypt_blocks(ks: aes_key_schedule, iv, d_in: int, d_out: int, nblocks: int, stream=None) -> None:
    ivp = _bytes_ptr(iv)
    _check(lib().aes_encrypt_blocks(ctypes.byref(ks), ivp[0] if ivp else None, d_in, d_out, nblocks,
                                    _stream_ptr(stream)))


def aes_decrypt_blocks(ks: aes_key_schedule, iv, d_in: int, d_out: int, nblocks: int, stream=None) -> None:
    ivp = _bytes_ptr(iv)
    _check(lib().aes_decrypt_blocks(ctypes.byref(ks), ivp[0] if ivp else None, d_in, d_out, nblocks,
                                    _stream_ptr(stream)))


def aes_crypt_host(ks: aes_key_schedule, iv, h_in: int, h_out: int, nblocks: int, dir, impl="auto",
                   stream=None) -> None:
    """Host-buffer variant: h_in / h_out are host addresses; returns when h_out is written."""
    ivp = _bytes_ptr(iv)
    _check(lib().aes_crypt_host(ctypes.byref(ks), ivp[0] if ivp else None, h_in, h_out, nblocks,
                                _dir(dir), _IMPLS[impl] if isinstance(impl, str) else int(impl),
                                _stream_ptr(stream)))


def aes_cbc_crypt(ks: aes_key_schedule, d_ivs: int, iv_per_msg: bool, d_in: int, d_out: int, nmsgs: int,
                  blocks_per_msg: int, dir, stream=None) -> None:
    """CBC over an nmsgs x blocks_per_msg matrix of blocks (device pointers)."""
    _check(lib().aes_cbc_crypt(ctypes.byref(ks), d_ivs, int(iv_per_msg), d_in, d_out, nmsgs, blocks_per_msg,
                               _dir(dir), _stream_ptr(stream)))


def cbc(x, ks: aes_key_schedule, ivs, dir="encrypt", out=None, stream=None):
    """CBC on a CUDA uint8 tensor of shape (nmsgs, 16 * blocks_per_msg); ivs is a CUDA uint8
    tensor of 16 bytes (one IV for all rows) or (nmsgs, 16) (one per row)."""
    import torch

    if x.dim() != 2 or x.shape[1] % 16 or x.dtype != torch.uint8 or not x.is_contiguous():
        raise ValueError("x must be a contiguous (nmsgs, 16*m) uint8 tensor")
    per_msg = ivs.numel() != 16
    if per_msg and tuple(ivs.shape) != (x.shape[0], 16):
        raise ValueError("ivs must hold 16 bytes or one 16-byte IV per row")
    if out is None:
        out = torch.empty_like(x)
    aes_cbc_crypt(ks, ivs.data_ptr(), per_msg, x.data_ptr(), out.data_ptr(), x.shape[0], x.shape[1] // 16, dir,
                  stream)
    return out


def aes_ctr_crypt(ks: aes_key_schedule, ctr0: bytes, d_in: int, d_out: int, nblocks: int, stream=None) -> None:
    p, _keep = _bytes_ptr(ctr0)
    _check(lib().aes_ctr_crypt(ctypes.byref(ks), p, d_in, d_out, nblocks, _stream_ptr(stream)))


def ctr(x, ks: aes_key_schedule, ctr0: bytes, out=None, stream=None):
    """Counter mode on a CUDA tensor of whole blocks (same call encrypts and decrypts)."""
    import torch

    n = _blocks_of(x)
    if out is None:
        out = torch.empty_like(x)
    aes_ctr_crypt(ks, ctr0, x.data_ptr(), out.data_ptr(), n, stream)
    return out


def aes_autotune_blocks(ks: aes_key_schedule, d_in: int, d_out: int, nblocks: int, dir, cache_path=None,
                        stream=None) -> dict:
    """Tunes AES_IMPL_AUTO for this device, direction and round count; returns the choice."""
    i, t, u = _I(), _I(), _I()
    cp = None if cache_path is None else str(cache_path).encode()
    _check(lib().aes_autotune_blocks(ctypes.byref(ks), d_in, d_out, nblocks, _dir(dir), cp, ctypes.byref(i),
                                     ctypes.byref(t), ctypes.byref(u), _stream_ptr(stream)))
    return {"impl": {AES_IMPL_TTABLE: "ttable", AES_IMPL_BITSLICE: "bitslice"}.get(i.value, i.value),
            "threads": t.value, "blocks_per_thread": u.value}


def aes_set_auto_choice(dir, nr: int, impl, threads: int, blocks_per_thread: int) -> None:
    """Sets (pins) the AES_IMPL_AUTO kernel for this device, direction and round count directly;
    impl "auto" clears it back to the default."""
    code = {"auto": AES_IMPL_AUTO, "ttable": AES_IMPL_TTABLE, "bitslice": AES_IMPL_BITSLICE}.get(impl, impl)
    _check(lib().aes_set_auto_choice(_dir(dir), nr, int(code), threads, blocks_per_thread))


def aes_gcm_workspace_bytes() -> int:
    return int(lib().aes_gcm_workspace_bytes())


def aes_gcm_crypt(ks: aes_key_schedule, iv: bytes, d_aad: int, aad_len: int, d_in: int, d_out: int, nbytes: int,
                  dir, d_tag: int, d_work: int, work_bytes: int, stream=None) -> None:
    p, _keep = _bytes_ptr(iv)
    _check(lib().aes_gcm_crypt(ctypes.byref(ks), p, len(iv), d_aad, aad_len, d_in, d_out, nbytes, _dir(dir), d_tag,
                               d_work, work_bytes, _stream_ptr(stream)))


def aes_gcm_decrypt_verify(ks: aes_key_schedule, iv: bytes, d_aad: int, aad_len: int, d_in: int, d_out: int,
                           nbytes: int, d_expected_tag: int, d_ok: int, d_tag: int, d_work: int, work_bytes: int,
                           stream=None) -> None:
    p, _keep = _bytes_ptr(iv)
    _check(lib().aes_gcm_decrypt_verify(ctypes.byref(ks), p, len(iv), d_aad, aad_len, d_in, d_out, nbytes,
                                        d_expected_tag, d_ok, d_tag, d_work, work_bytes, _stream_ptr(stream)))


def gcm_open(x, ks: aes_key_schedule, iv: bytes, tag, aad=None, out=None, stream=None):
    """AES-GCM decryption of the CUDA uint8 tensor x with the received 16-byte `tag` (CUDA
    tensor) checked on the device; returns (plaintext, ok) with ok a CUDA int32 tensor holding
    1 if the tag matched, else 0.  Use the plaintext only when ok is 1."""
    import torch

    if x.dtype != torch.uint8 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA uint8 tensor")
    if tag.dtype != torch.uint8 or not tag.is_cuda or tag.numel() != 16:
        raise ValueError("tag must be 16 bytes in a CUDA uint8 tensor")
    if out is None:
        out = torch.empty_like(x)
    ok = torch.empty(1, dtype=torch.int32, device=x.device)
    computed = torch.empty(16, dtype=torch.uint8, device=x.device)
    work = torch.empty(aes_gcm_workspace_bytes(), dtype=torch.uint8, device=x.device)
    a_ptr, a_len = (aad.data_ptr(), aad.numel()) if aad is not None and aad.numel() else (None, 0)
    aes_gcm_decrypt_verify(ks, iv, a_ptr, a_len, x.data_ptr() if x.numel() else None,
                           out.data_ptr() if x.numel() else None, x.numel(), tag.data_ptr(), ok.data_ptr(),
                           computed.data_ptr(), work.data_ptr(), work.numel(), stream)
    if isinstance(stream, torch.cuda.Stream):  # the scratch tensors are freed here, still in use there
        for t in (work, computed):
            t.record_stream(stream)
    return out, ok


def gcm(x, ks: aes_key_schedule, iv: bytes, aad=None, dir="encrypt", out=None, stream=None):
    """AES-GCM on a contiguous CUDA uint8 tensor of any length; returns (output, 16-byte tag
    tensor on the device).  On decryption the tag is the one computed from `x`: compare it
    with the received tag before using the output."""
    import torch

    if x.dtype != torch.uint8 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA uint8 tensor")
    if out is None:
        out = torch.empty_like(x)
    tag = torch.empty(16, dtype=torch.uint8, device=x.device)
    work = torch.empty(aes_gcm_workspace_bytes(), dtype=torch.uint8, device=x.device)
    a_ptr, a_len = (aad.data_ptr(), aad.numel()) if aad is not None and aad.numel() else (None, 0)
    aes_gcm_crypt(ks, iv, a_ptr, a_len, x.data_ptr() if x.numel() else None, out.data_ptr() if x.numel() else None,
                  x.numel(), dir, tag.data_ptr(), work.data_ptr(), work.numel(), stream)
    if isinstance(stream, torch.cuda.Stream):  # the workspace is freed here, still in use there
        work.record_stream(stream)
    return out, tag


def aes_scan_equal(d_column: int, nrecords: int, needle: bytes, d_matches: int, max_matches: int, d_count: int,
                   stream=None) -> None:
    p, _keep = _bytes_ptr(needle)
    _check(lib().aes_scan_equal(d_column, nrecords, p, d_matches, max_matches, d_count, _stream_ptr(stream)))


def find_equal(column, needle: bytes, max_matches: int = 1 << 20, stream=None):
    """Indices (sorted) of the 16-byte records of the CUDA tensor `column` equal to `needle`."""
    import torch

    n = _blocks_of(column)
    matches = torch.empty(max(1, max_matches), dtype=torch.int64, device=column.device)
    count = torch.zeros(1, dtype=torch.int64, device=column.device)
    aes_scan_equal(column.data_ptr(), n, needle, matches.data_ptr(), max_matches, count.data_ptr(), stream)
    k = int(count.item())
    return torch.sort(matches[: min(k, max_matches)]).values, k


def aes_crypt_batched_noalloc(schedules, msgs, d_in: int, d_out: int, buf_bytes: int, stream=None) -> None:
    """Allocation-free batched call: `schedules` is a ctypes array of aes_key_schedule."""
    a, p, n = _msgs_ptr(msgs)
    _check(lib().aes_crypt_batched_noalloc(schedules, len(schedules), p, n, d_in, d_out, buf_bytes,
                                           _stream_ptr(stream)))


# ---- key pool and batches -------------------------------------------------------------------

def _msgs_ptr(msgs):
    """msgs: numpy array of msg_dtype() (or a list of (key_idx, dir, offset, length))."""
    import numpy as np
    dt = msg_dtype()
    if isinstance(msgs, np.ndarray) and msgs.dtype == dt and msgs.flags["C_CONTIGUOUS"]:
        a = msgs
    else:
        a = np.ascontiguousarray(msgs if isinstance(msgs, np.ndarray) else np.array(msgs, dtype=dt), dtype=dt)
    return a, a.ctypes.data, a.shape[0]


class KeyPool:
    """Device-resident key schedules (aes_keypool_*)."""

    def __init__(self, capacity: int):
        h = _VP()
        _check(lib().aes_keypool_create(capacity, ctypes.byref(h)))
        self.handle = h
        self.capacity = capacity

    def load_keys(self, first: int, keys, key_bits: int, stream=None) -> None:
        """Expand len(keys) raw keys (uint8 array, key_bits/8 bytes each) on the device."""
        import numpy as np
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8).reshape(-1))
        count = k.size // (key_bits // 8)
        _check(lib().aes_keypool_load_keys(self.handle, first, count, k.ctypes.data_as(_U8P), key_bits,
                                           _stream_ptr(stream)))

    def set(self, idx: int, ks: aes_key_schedule) -> None:
        _check(lib().aes_keypool_set(self.handle, idx, ctypes.byref(ks)))

    def rounds(self, idx: int) -> int:
        return lib().aes_keypool_rounds(self.handle, idx)

    def close(self) -> None:
        if self.handle:
            _check(lib().aes_keypool_destroy(self.handle))
            self.handle = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """A reusable batched-launch context (aes_batch_*)."""

    def __init__(self, pool: KeyPool, max_msgs: int):
        h = _VP()
        _check(lib().aes_batch_create(pool.handle, max_msgs, ctypes.byref(h)))
        self.handle, self.pool = h, pool

    def run(self, msgs, d_in: int, d_out: int, buf_bytes: int, stream=None, ivs=None) -> None:
        """ivs: None, or a host uint8 array of len(msgs) x 16 bytes (one IV per message)."""
        a, p, n = _msgs_ptr(msgs)
        if ivs is None:
            _check(lib().aes_batch_run(self.handle, p, n, d_in, d_out, buf_bytes, _stream_ptr(stream)))
        else:
            v = _ivs_array(ivs, n)
            _check(lib().aes_batch_run_iv(self.handle, p, v.ctypes.data, n, d_in, d_out, buf_bytes,
                                          _stream_ptr(stream)))

    def autotune(self, msgs, d_in: int, d_out: int, buf_bytes: int, cache_path: str | None = None,
                 stream=None) -> tuple[int, int]:
        a, p, n = _msgs_ptr(msgs)
        t, u = ctypes.c_int(), ctypes.c_int()
        _check(lib().aes_batch_autotune(self.handle, p, n, d_in, d_out, buf_bytes,
                                        cache_path.encode() if cache_path else None, ctypes.byref(t),
                                        ctypes.byref(u), _stream_ptr(stream)))
        return t.value, u.value

    def set_shape(self, threads: int, blocks_per_lane: int) -> None:
        _check(lib().aes_batch_set_shape(self.handle, threads, blocks_per_lane))

    def close(self) -> None:
        if self.handle:
            _check(lib().aes_batch_destroy(self.handle))
            self.handle = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def aes_crypt_batched(pool: KeyPool, msgs, d_in: int, d_out: int, buf_bytes: int, stream=None) -> None:
    a, p, n = _msgs_ptr(msgs)
    _check(lib().aes_crypt_batched(pool.handle, p, n, d_in, d_out, buf_bytes, _stream_ptr(stream)))


def _ivs_array(ivs, n: int):
    import numpy as np
    v = np.ascontiguousarray(np.asarray(ivs, dtype=np.uint8).reshape(-1))
    if v.size != 16 * n:
        raise ValueError("ivs must hold 16 bytes per message")
    return v


def aes_cbc_batched(pool: KeyPool, msgs, ivs, d_in: int, d_out: int, buf_bytes: int, stream=None) -> None:
    """CBC chained over each message (its own key slot and IV; ivs: host uint8, len(msgs) x 16,
    or None for zero IVs)."""
    a, p, n = _msgs_ptr(msgs)
    v = None if ivs is None else _ivs_array(ivs, n)
    _check(lib().aes_cbc_batched(pool.handle, p, None if v is None else v.ctypes.data, n, d_in, d_out, buf_bytes,
                                 _stream_ptr(stream)))


def aes_crypt_batched_iv(pool: KeyPool, msgs, ivs, d_in: int, d_out: int, buf_bytes: int, stream=None) -> None:
    """aes_crypt_batched with one 16-byte IV per message (ivs: host uint8, len(msgs) x 16)."""
    a, p, n = _msgs_ptr(msgs)
    v = _ivs_array(ivs, n)
    _check(lib().aes_crypt_batched_iv(pool.handle, p, v.ctypes.data, n, d_in, d_out, buf_bytes, _stream_ptr(stream)))


# ---- server -----------------------------------------------------------------------------------

class Server:
    """Continuous-batching request server (aes_server_*)."""

    def __init__(self, pool: KeyPool, hbm_budget: int = 1 << 30, max_inflight: int = 1 << 16, nstreams: int = 4,
                 max_batch: int = 4096, queue_capacity: int = 1 << 16, fail_every: int = 0, linger_us: int = 0):
        cfg = aes_server_cfg(hbm_budget, max_inflight, nstreams, max_batch, queue_capacity, fail_every, linger_us)
        h = _VP()
        _check(lib().aes_server_create(ctypes.byref(cfg), pool.handle, ctypes.byref(h)))
        self.handle, self.pool = h, pool

    def submit(self, key_idx: int, dir, src: int, dst: int, length: int, src_on_device: bool,
               dst_on_device: bool) -> int:
        r = aes_request(key_idx, _dir(dir), src, dst, length, int(src_on_device), int(dst_on_device))
        t = ctypes.c_uint64()
        _check(lib().aes_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def submit_many(self, reqs) -> "np.ndarray":
        """Queue a numpy array of request_dtype() all at once; returns the tickets (uint64)."""
        import numpy as np
        a = np.ascontiguousarray(reqs, dtype=request_dtype())
        t = np.empty(a.shape[0], dtype=np.uint64)
        _check(lib().aes_server_submit_many(self.handle, a.ctypes.data, a.shape[0], t.ctypes.data))
        return t

    def try_submit(self, *args, **kw) -> int | None:
        """submit(), or None when the queue is full (AES_EAGAIN)."""
        try:
            return self.submit(*args, **kw)
        except AesError as e:
            if e.status == AES_EAGAIN:
                return None
            raise

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        """AES_REQ_DONE / AES_REQ_FAILED, or AES_REQ_PENDING when the wait ran out."""
        st = ctypes.c_int()
        rc = lib().aes_server_poll(self.handle, ticket, timeout_us, ctypes.byref(st))
        if rc == AES_ETIMEDOUT:
            return AES_REQ_PENDING
        _check(rc)
        return st.value

    def stats(self) -> dict:
        out = aes_stats()
        _check(lib().aes_server_stats(self.handle, ctypes.byref(out)))
        return out.as_dict()

    def reset_stats(self) -> None:
        _check(lib().aes_server_stats_reset(self.handle))

    def close(self) -> None:
        if self.handle:
            _check(lib().aes_server_destroy(self.handle))
            self.handle = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- torch conveniences (still one C call each) -------------------------------------------

def _blocks_of(t) -> int:
    if t.dtype.itemsize * t.numel() % 16:
        raise ValueError("tensor size must be a whole number of 16-byte blocks")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensor must be a contiguous CUDA tensor")
    return t.numel() * t.dtype.itemsize // 16


def crypt(x, ks: aes_key_schedule, dir="encrypt", iv=None, out=None, impl="auto", stream=None):
    """Encrypt or decrypt the CUDA tensor `x` (whole 16-byte blocks) into `out` (new if None)."""
    import torch

    n = _blocks_of(x)
    if out is None:
        out = torch.empty_like(x)
    elif _blocks_of(out) != n:
        raise ValueError("out has a different size")
    aes_crypt_blocks(ks, iv, x.data_ptr(), out.data_ptr(), n, dir, impl, stream)
    return out


def encrypt(x, ks, iv=None, out=None, impl="auto", stream=None):
    return crypt(x, ks, "encrypt", iv, out, impl, stream)


def decrypt(x, ks, iv=None, out=None, impl="auto", stream=None):
    return crypt(x, ks, "decrypt", iv, out, impl, stream)


def build(verbose: bool = False):
    """Compile libaesgb.so in-tree (see builder.py)."""
    from . import builder
    return builder.build(verbose=verbose)
