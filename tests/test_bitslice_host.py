"""The bitsliced kernel's round code (aes_bitslice.cuh: bit-plane transposes, the generated
S-box networks, MixColumns with the round key folded in, InvMixColumns as MixColumns o P, the
masks built on the host) compiled as plain host C++ and run on the CPU, against the oracle:
every key size, with and without IV, both directions, ragged block counts.  The same source
runs in the CUDA kernel, so a mistake in the circuits or the key folding shows here without
a GPU."""
import ctypes
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_1506_08503_gb300" / "csrc"


@pytest.fixture(scope="module")
def host_bs(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = tmp_path_factory.mktemp("bs") / "libbs_host.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-w", "-I", str(ROOT / "include"), "-I", str(CSRC),
                    "-o", str(out), str(ROOT / "tests" / "host" / "bitslice_host.cpp")], check=True,
                   capture_output=True, text=True)
    lib = ctypes.CDLL(str(out))
    lib.bs_host_crypt.restype = ctypes.c_int
    lib.bs_host_crypt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_size_t]
    return lib


def _crypt(lib, aes, key, bits, direction, data, iv):
    ks = aes.aes_key_expand(key.tobytes(), bits)
    out = np.empty_like(data)
    ivb = None if iv is None else (ctypes.c_uint8 * 16).from_buffer_copy(iv.tobytes())
    rc = lib.bs_host_crypt(ctypes.addressof(ks), direction, ctypes.addressof(ivb) if ivb is not None else None,
                           data.ctypes.data, out.ctypes.data, data.size // 16)
    assert rc == 0
    return out


@pytest.mark.parametrize("bits", [128, 192, 256])
@pytest.mark.parametrize("with_iv", [False, True])
def test_host_tile_matches_oracle(host_bs, aes, orc, bits, with_iv):
    rng = np.random.default_rng(bits + 7 * with_iv)
    for n in (1, 31, 32, 33, 95):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8) if with_iv else None
        data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
        ct = _crypt(host_bs, aes, key, bits, 0, data, iv)
        assert np.array_equal(ct, orc.encrypt_blocks(key, data, iv=iv)), n
        pt = _crypt(host_bs, aes, key, bits, 1, data, iv)  # decryption of arbitrary data
        assert np.array_equal(pt, orc.decrypt_blocks(key, data, iv=iv)), n
        assert np.array_equal(_crypt(host_bs, aes, key, bits, 1, ct, iv), data)


def test_host_tile_special_blocks(host_bs, aes, orc):
    """All-zero and all-one keys and blocks (every mask plane 0 or all ones)."""
    for key in (np.zeros(16, np.uint8), np.full(16, 255, np.uint8), np.zeros(32, np.uint8)):
        data = np.concatenate([np.zeros(16 * 16, np.uint8), np.full(16 * 16, 255, np.uint8)])
        ct = _crypt(host_bs, aes, key, 8 * key.size, 0, data, None)
        assert np.array_equal(ct, orc.encrypt_blocks(key, data))
