"""ctypes wrapper of the CPU oracle (aes_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the CPU
baseline leg of bench.py, never by the product package.  It shares no code with the CUDA
library and imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "aes_oracle.c"
HDR = HERE / "aes_oracle.h"
LIB = HERE / "liboracle.so"

_lock = threading.Lock()
_lib = None

_U8P = ctypes.POINTER(ctypes.c_uint8)


def build(src: Path = SRC, out: Path = LIB, extra: tuple[str, ...] = ()) -> Path:
    """Compile the oracle with gcc (plain C11, pthreads)."""
    newest = max(src.stat().st_mtime, HDR.stat().st_mtime)
    if out.exists() and out.stat().st_mtime >= newest and not extra:
        return out
    tmp = out.with_name(out.name + f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-I", str(HERE),
           *extra, "-o", str(tmp), str(src), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def load(path: Path | None = None) -> ctypes.CDLL:
    """Load (building if needed) the oracle library; `path` loads a specific build."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(str(path)))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(str(build())))
        return _lib


def _declare(l: ctypes.CDLL) -> ctypes.CDLL:
    u8, i, sz = ctypes.c_uint8, ctypes.c_int, ctypes.c_size_t
    sig = {
        "oracle_gf_add": (u8, [u8, u8]),
        "oracle_gf_mul": (u8, [u8, u8]),
        "oracle_gf_inv": (u8, [u8]),
        "oracle_affine": (u8, [u8]),
        "oracle_inv_affine": (u8, [u8]),
        "oracle_sbox": (u8, [u8]),
        "oracle_inv_sbox": (u8, [u8]),
        "oracle_sub_bytes": (None, [_U8P]),
        "oracle_inv_sub_bytes": (None, [_U8P]),
        "oracle_shift_rows": (None, [_U8P]),
        "oracle_inv_shift_rows": (None, [_U8P]),
        "oracle_mix_columns": (None, [_U8P]),
        "oracle_inv_mix_columns": (None, [_U8P]),
        "oracle_add": (None, [_U8P, _U8P]),
        "oracle_rcon": (u8, [i]),
        "oracle_key_expand": (i, [_U8P, i, _U8P]),
        "oracle_key_expand_words": (i, [_U8P, i, _U8P]),
        "oracle_encrypt_block": (None, [_U8P, i, _U8P, _U8P, _U8P]),
        "oracle_decrypt_block": (None, [_U8P, i, _U8P, _U8P, _U8P]),
        "oracle_encrypt_blocks": (i, [_U8P, i, _U8P, _U8P, _U8P, sz, i]),
        "oracle_decrypt_blocks": (i, [_U8P, i, _U8P, _U8P, _U8P, sz, i]),
        "oracle_cbc_encrypt": (None, [_U8P, i, _U8P, _U8P, _U8P, sz]),
        "oracle_cbc_decrypt": (None, [_U8P, i, _U8P, _U8P, _U8P, sz]),
        "oracle_ctr_crypt": (None, [_U8P, i, _U8P, _U8P, _U8P, sz]),
        "oracle_gf128_mul": (None, [_U8P, _U8P, _U8P]),
        "oracle_ghash": (None, [_U8P, _U8P, sz, _U8P]),
        "oracle_gcm_crypt": (None, [_U8P, i, _U8P, _U8P, sz, _U8P, _U8P, sz, i, _U8P]),
        "oracle_gcm_crypt_iv": (None, [_U8P, i, _U8P, sz, _U8P, sz, _U8P, _U8P, sz, i, _U8P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(l, name)
        f.restype, f.argtypes = res, args
    return l


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_U8P)


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.frombuffer(bytes(x), dtype=np.uint8) if isinstance(x, (bytes, bytearray)) else x,
                                dtype=np.uint8)


class Oracle:
    """numpy-facing view of one oracle build."""

    def __init__(self, lib: ctypes.CDLL | None = None):
        self.lib = lib or load()

    # field and S-box
    def gf_mul(self, a: int, b: int) -> int: return self.lib.oracle_gf_mul(a, b)
    def gf_add(self, a: int, b: int) -> int: return self.lib.oracle_gf_add(a, b)
    def gf_inv(self, a: int) -> int: return self.lib.oracle_gf_inv(a)
    def sbox(self, x: int) -> int: return self.lib.oracle_sbox(x)
    def inv_sbox(self, x: int) -> int: return self.lib.oracle_inv_sbox(x)
    def affine(self, x: int) -> int: return self.lib.oracle_affine(x)
    def inv_affine(self, x: int) -> int: return self.lib.oracle_inv_affine(x)
    def rcon(self, r: int) -> int: return self.lib.oracle_rcon(r)

    def sbox_table(self) -> np.ndarray:
        return np.array([self.sbox(x) for x in range(256)], dtype=np.uint8)

    def inv_sbox_table(self) -> np.ndarray:
        return np.array([self.inv_sbox(x) for x in range(256)], dtype=np.uint8)

    # one-state steps (return a new array)
    def _step(self, name: str, s) -> np.ndarray:
        a = _u8(s).copy()
        getattr(self.lib, name)(_p(a))
        return a

    def sub_bytes(self, s): return self._step("oracle_sub_bytes", s)
    def inv_sub_bytes(self, s): return self._step("oracle_inv_sub_bytes", s)
    def shift_rows(self, s): return self._step("oracle_shift_rows", s)
    def inv_shift_rows(self, s): return self._step("oracle_inv_shift_rows", s)
    def mix_columns(self, s): return self._step("oracle_mix_columns", s)
    def inv_mix_columns(self, s): return self._step("oracle_inv_mix_columns", s)

    # keys
    def key_expand(self, key, key_bits: int | None = None) -> tuple[np.ndarray, int]:
        k = _u8(key)
        key_bits = key_bits or 8 * k.size
        out = np.zeros(16 * 15, dtype=np.uint8)
        nr = self.lib.oracle_key_expand(_p(k), key_bits, _p(out))
        if nr < 0:
            raise ValueError(f"bad key size {key_bits}")
        return out[: 16 * (nr + 1)].copy(), nr

    def key_expand_words(self, key, nk: int) -> tuple[np.ndarray, int]:
        k = _u8(key)
        out = np.zeros(16 * 15, dtype=np.uint8)
        nr = self.lib.oracle_key_expand_words(_p(k), nk, _p(out))
        if nr < 0:
            raise ValueError(f"bad nk {nk}")
        return out[: 16 * (nr + 1)].copy(), nr

    # many blocks
    def _blocks(self, fn: str, key, data, iv=None, threads: int = 1) -> np.ndarray:
        rk, nr = self.key_expand(key)
        src = _u8(data).reshape(-1)
        if src.size % 16:
            raise ValueError("data must be whole 16-byte blocks")
        out = np.empty_like(src)
        ivv = None if iv is None else _u8(iv)
        getattr(self.lib, fn)(_p(rk), nr, _p(ivv), _p(src), _p(out), src.size // 16, threads)
        return out

    def encrypt_blocks(self, key, data, iv=None, threads: int = 1) -> np.ndarray:
        return self._blocks("oracle_encrypt_blocks", key, data, iv, threads)

    def decrypt_blocks(self, key, data, iv=None, threads: int = 1) -> np.ndarray:
        return self._blocks("oracle_decrypt_blocks", key, data, iv, threads)

    def cbc_encrypt(self, key, iv, data) -> np.ndarray:
        rk, nr = self.key_expand(key)
        src = _u8(data).reshape(-1)
        out = np.empty_like(src)
        self.lib.oracle_cbc_encrypt(_p(rk), nr, _p(_u8(iv)), _p(src), _p(out), src.size // 16)
        return out

    def cbc_decrypt(self, key, iv, data) -> np.ndarray:
        rk, nr = self.key_expand(key)
        src = _u8(data).reshape(-1)
        out = np.empty_like(src)
        self.lib.oracle_cbc_decrypt(_p(rk), nr, _p(_u8(iv)), _p(src), _p(out), src.size // 16)
        return out

    def ctr_crypt(self, key, ctr0, data) -> np.ndarray:
        rk, nr = self.key_expand(key)
        src = _u8(data).reshape(-1)
        out = np.empty_like(src)
        self.lib.oracle_ctr_crypt(_p(rk), nr, _p(_u8(ctr0)), _p(src), _p(out), src.size // 16)
        return out

    # Galois/Counter Mode
    def gf128_mul(self, x, y) -> np.ndarray:
        z = np.empty(16, dtype=np.uint8)
        self.lib.oracle_gf128_mul(_p(_u8(x)), _p(_u8(y)), _p(z))
        return z

    def ghash(self, h, data) -> np.ndarray:
        src = _u8(data).reshape(-1)
        if src.size % 16:
            raise ValueError("GHASH input must be whole 16-byte blocks")
        y = np.empty(16, dtype=np.uint8)
        self.lib.oracle_ghash(_p(_u8(h)), _p(src), src.size // 16, _p(y))
        return y

    def gcm_crypt(self, key, iv, data, aad=b"", decrypt: bool = False) -> tuple[np.ndarray, np.ndarray]:
        """(output bytes, tag); the data and AAD may have any length."""
        rk, nr = self.key_expand(key)
        ivv = _u8(iv).reshape(-1)
        if ivv.size == 0:
            raise ValueError("a GCM IV has at least one byte")
        src = _u8(data).reshape(-1)
        a = _u8(aad).reshape(-1)
        out = np.empty_like(src)
        tag = np.empty(16, dtype=np.uint8)
        self.lib.oracle_gcm_crypt_iv(_p(rk), nr, _p(ivv), ivv.size, _p(a) if a.size else None, a.size,
                                     _p(src) if src.size else None, _p(out) if src.size else None, src.size,
                                     int(decrypt), _p(tag))
        return out, tag


_default: Oracle | None = None


def oracle() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
