"""The C ABI on the host, no GPU needed: the library loads, exports every function that
include/*.h declares, expands keys exactly like the oracle, and rejects bad arguments before
any CUDA call."""
import ctypes
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions() -> set[str]:
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(aes_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_core_entry_points():
    names = declared_functions()
    for n in ("aes_key_expand", "aes_encrypt_blocks", "aes_decrypt_blocks", "aes_crypt_blocks", "aes_last_error"):
        assert n in names
    # the boundary's key-pool, batched and server calls under their contract names
    for n in ("aes_keypool_create", "aes_keypool_set", "aes_keypool_destroy", "aes_crypt_batched",
              "aes_server_create", "aes_server_submit", "aes_server_poll", "aes_server_stats", "aes_server_destroy"):
        assert n in names, n


def test_library_exports_every_declared_symbol(aes):
    lib = aes.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", str(aes.LIB_PATH)], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = sorted(n for n in declared_functions() if n not in exported)
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None
    # the Python binding mirrors the same names
    assert set(aes.declared_symbols()) <= declared_functions()


@pytest.mark.parametrize("bits", [128, 192, 256])
def test_key_expand_matches_oracle(aes, orc, bits):
    rng = np.random.default_rng(bits)
    for _ in range(200):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
        ks = aes.aes_key_expand(key.tobytes(), bits)
        rk, nr = orc.key_expand(key, bits)
        assert ks.nr == nr
        assert ks.round_keys() == rk.tobytes()
        tail = bytes(bytearray(ks.rk))[16 * (nr + 1):]
        assert tail == bytes(len(tail))


def test_key_expand_rejects_bad_sizes(aes):
    ks = aes.aes_key_schedule()
    key = (ctypes.c_uint8 * 32)()
    for bits in (0, 64, 160, 512, -128):
        assert aes.lib().aes_key_expand(key, bits, ctypes.byref(ks)) == aes.AES_EINVAL
        assert "key_bits" in aes.aes_last_error()
    assert aes.lib().aes_key_expand(None, 128, ctypes.byref(ks)) == aes.AES_EINVAL
    assert aes.lib().aes_key_expand(key, 128, None) == aes.AES_EINVAL


def test_crypt_argument_checks_before_any_cuda_call(aes):
    lib = aes.lib()
    ks = aes.aes_key_expand(bytes(16))
    kp = ctypes.byref(ks)
    base = 1 << 40  # never dereferenced: every call below fails validation first
    assert lib.aes_crypt_blocks(kp, None, base, base + 4096, 0, 0, 0, None) == aes.AES_OK  # empty
    assert lib.aes_crypt_blocks(kp, None, base + 8, base + 4096, 4, 0, 0, None) == aes.AES_EINVAL  # misaligned
    assert lib.aes_crypt_blocks(kp, None, base, base + 16, 4, 0, 0, None) == aes.AES_EINVAL  # partial overlap
    assert lib.aes_crypt_blocks(kp, None, None, base, 4, 0, 0, None) == aes.AES_EINVAL
    assert lib.aes_crypt_blocks(kp, None, base, base + 4096, 4, 2, 0, None) == aes.AES_EINVAL  # bad dir
    assert lib.aes_crypt_blocks(kp, None, base, base + 4096, 4, 0, 9, None) == aes.AES_EINVAL  # bad impl
    assert lib.aes_crypt_blocks(kp, None, base, base + 4096, 1 << 62, 0, 0, None) == aes.AES_EINVAL  # too big
    bad = aes.aes_key_schedule()
    bad.nr = 11
    assert lib.aes_crypt_blocks(ctypes.byref(bad), None, base, base + 4096, 4, 0, 0, None) == aes.AES_EINVAL
    assert lib.aes_crypt_blocks(None, None, base, base + 4096, 4, 0, 0, None) == aes.AES_EINVAL
    assert aes.aes_last_error()


def test_binding_raises_with_message(aes):
    ks = aes.aes_key_expand(bytes(16))
    with pytest.raises(aes.AesError) as ei:
        aes.aes_crypt_blocks(ks, None, (1 << 40) + 8, 1 << 41, 4, "encrypt")
    assert ei.value.status == aes.AES_EINVAL and "aligned" in str(ei.value)


def test_pool_and_batch_null_handling_without_gpu(aes):
    lib = aes.lib()
    h = ctypes.c_void_p()
    assert lib.aes_keypool_create(0, ctypes.byref(h)) == aes.AES_EINVAL
    assert lib.aes_keypool_create(1 << 30, ctypes.byref(h)) == aes.AES_EINVAL
    assert lib.aes_keypool_create(16, None) == aes.AES_EINVAL
    assert lib.aes_keypool_destroy(None) == aes.AES_OK
    assert lib.aes_keypool_rounds(None, 0) == 0
    assert lib.aes_batch_create(None, 16, ctypes.byref(h)) == aes.AES_EINVAL
    assert lib.aes_batch_destroy(None) == aes.AES_OK
    assert lib.aes_batch_run(None, None, 0, None, None, 0, None) == aes.AES_EINVAL
    assert lib.aes_batch_set_shape(None, 512, 4) == aes.AES_EINVAL
    assert lib.aes_crypt_batched(None, None, 0, None, None, 0, None) == aes.AES_EINVAL
    assert lib.aes_crypt_host(None, None, None, None, 4, 0, 0, None) == aes.AES_EINVAL


def test_message_struct_layout(aes):
    assert ctypes.sizeof(aes.aes_msg) == 24 == aes.msg_dtype().itemsize
    assert ctypes.sizeof(aes.aes_key_schedule) == 4 + 15 * 16


def test_gcm_argument_checks_before_any_cuda_call(aes):
    lib = aes.lib()
    ks = aes.aes_key_expand(bytes(16))
    kp = ctypes.byref(ks)
    iv = (ctypes.c_uint8 * 300)()
    base = 1 << 40  # never dereferenced
    W = aes.aes_gcm_workspace_bytes()
    assert W >= 256 * 16  # a partial sum per CTA and the finished-CTA ticket
    work, tag = base + (1 << 30), base + (1 << 31)

    def call(iv_len=12, aad=None, aad_len=0, src=base, dst=base, n=64, d=0, t=tag, w=work, wb=W):
        return lib.aes_gcm_crypt(kp, iv, iv_len, aad, aad_len, src, dst, n, d, t, w, wb, None)

    for iv_len in (0, 257):
        assert call(iv_len=iv_len) == aes.AES_EINVAL and "IV" in aes.aes_last_error()
    assert call(wb=W - 16) == aes.AES_EINVAL  # workspace too small
    assert call(w=work + 8) == aes.AES_EINVAL  # workspace misaligned
    assert call(w=base + 32) == aes.AES_EINVAL  # workspace overlaps the data
    assert call(t=None) == aes.AES_EINVAL
    assert call(d=3) == aes.AES_EINVAL
    assert call(src=base + 8) == aes.AES_EINVAL  # misaligned data
    assert call(dst=base + 16) == aes.AES_EINVAL  # partial overlap
    assert call(aad=None, aad_len=5) == aes.AES_EINVAL

    # decryption with the tag check: the expected tag and the ok flag are required and must not
    # overlap what the call writes
    lib.aes_gcm_decrypt_verify.restype = ctypes.c_int
    exp_tag, ok = base + (1 << 32), base + (1 << 33)

    def verify(e=exp_tag, o=ok, t=tag, src=base, dst=base):
        return lib.aes_gcm_decrypt_verify(kp, iv, 12, None, 0, src, dst, 64, e, o, t, work, W, None)

    assert verify(e=None) == aes.AES_EINVAL and "expected tag" in aes.aes_last_error()
    assert verify(o=None) == aes.AES_EINVAL
    assert verify(o=ok + 2) == aes.AES_EINVAL  # ok flag not int-aligned
    assert verify(o=tag + 4) == aes.AES_EINVAL  # ok flag inside the tag
    assert verify(e=base + 16) == aes.AES_EINVAL  # expected tag inside the output
    assert verify(o=work + 64) == aes.AES_EINVAL  # ok flag inside the workspace
    assert call(aad=base + 48, aad_len=32) == aes.AES_EINVAL  # output overlaps the AAD
    assert call(n=16 * (1 << 32)) == aes.AES_EINVAL  # beyond 2^32 - 2 blocks
    assert call(src=None, dst=None) == aes.AES_EINVAL


def test_autotune_argument_checks_before_any_cuda_call(aes):
    lib = aes.lib()
    ks = aes.aes_key_expand(bytes(16))
    kp = ctypes.byref(ks)
    base = 1 << 40  # never dereferenced
    assert lib.aes_autotune_blocks(kp, base, base + 4096, 0, 0, None, None, None, None, None) == aes.AES_EINVAL
    assert lib.aes_autotune_blocks(kp, base, base + 4096, 4, 2, None, None, None, None, None) == aes.AES_EINVAL
    assert lib.aes_autotune_blocks(kp, base + 8, base + 4096, 4, 0, None, None, None, None, None) == aes.AES_EINVAL
    assert lib.aes_autotune_blocks(kp, base, base + 16, 4, 0, None, None, None, None, None) == aes.AES_EINVAL
    assert lib.aes_autotune_blocks(None, base, base + 4096, 4, 0, None, None, None, None, None) == aes.AES_EINVAL


def test_set_auto_choice_validates_before_any_cuda_call(aes):
    lib = aes.lib()
    assert lib.aes_set_auto_choice(2, 10, aes.AES_IMPL_TTABLE, 512, 2) == aes.AES_EINVAL  # bad dir
    assert lib.aes_set_auto_choice(0, 11, aes.AES_IMPL_TTABLE, 512, 2) == aes.AES_EINVAL  # bad nr
    assert lib.aes_set_auto_choice(0, 10, aes.AES_IMPL_TTABLE, 500, 2) == aes.AES_EINVAL  # not compiled
    assert lib.aes_set_auto_choice(0, 10, 7, 512, 2) == aes.AES_EINVAL
