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
                                  _DIRS[dir], _IMPLS[impl] if isinstance(impl, str) else int(impl),
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
                                _DIRS[dir], _IMPLS[impl] if isinstance(impl, str) else int(impl),
                                _stream_ptr(stream)))


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
