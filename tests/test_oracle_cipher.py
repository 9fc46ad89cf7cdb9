"""Pins for the oracle's round steps, key schedules and cipher (paper Section II, App. A1,
A3, A4).

The strongest pin is bit-exact agreement with OpenSSL's AES (through the `cryptography`
package), an implementation that shares nothing with the oracle: ECB for AES-128/192/256
over many random keys and blocks, and CBC (the paper's mode) for one-block and multi-block
messages.  The step tests tie the paper's printed constants to definitions that do not come
from the paper.
"""
from pathlib import Path

import numpy as np
import pytest

from test_oracle_field import np_field_mul

CONST = Path(__file__).parent / "golden" / "paper_constants.txt"


def _const(name):
    for line in CONST.read_text().splitlines():
        if line.startswith(name + " "):
            return [int(v) for v in line.split()[1:]]
    raise KeyError(name)


def _openssl():
    return pytest.importorskip("cryptography.hazmat.primitives.ciphers")


def openssl_ecb(key: bytes, data: bytes, decrypt: bool = False) -> bytes:
    c = _openssl()
    cipher = c.Cipher(c.algorithms.AES(key), c.modes.ECB())
    op = cipher.decryptor() if decrypt else cipher.encryptor()
    return op.update(data) + op.finalize()


def openssl_cbc(key: bytes, iv: bytes, data: bytes, decrypt: bool = False) -> bytes:
    c = _openssl()
    cipher = c.Cipher(c.algorithms.AES(key), c.modes.CBC(iv))
    op = cipher.decryptor() if decrypt else cipher.encryptor()
    return op.update(data) + op.finalize()


# ---- round steps ---------------------------------------------------------------------------

def test_shift_rows_is_row_rotation(orc):
    # AES definition: row r of the state rotates left by r; byte index = r + 4c
    s = np.arange(16, dtype=np.uint8)
    out = orc.shift_rows(s)
    for r in range(4):
        for c in range(4):
            assert out[r + 4 * c] == s[r + 4 * ((c + r) % 4)]
    back = orc.inv_shift_rows(out)
    assert (back == s).all()


def test_paper_shift_rows_lists_match_rotation():
    dst, src, isrc = _const("shiftrows_dst"), _const("shiftrows_src"), _const("inv_shiftrows_src")
    for d, s_, si in zip(dst, src, isrc):
        r, c = (d - 1) % 4, (d - 1) // 4
        assert s_ - 1 == r + 4 * ((c + r) % 4)
        assert si - 1 == r + 4 * ((c - r) % 4)


def test_mix_matrices_are_inverse_over_gf():
    row, irow = _const("mix_row"), _const("inv_mix_row")
    m = [[row[(j - i) % 4] for j in range(4)] for i in range(4)]
    mi = [[irow[(j - i) % 4] for j in range(4)] for i in range(4)]
    for i in range(4):
        for j in range(4):
            acc = 0
            for k in range(4):
                acc ^= np_field_mul(m[i][k], mi[k][j])
            assert acc == (1 if i == j else 0)


def test_mix_columns_round_trip_and_linearity(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.integers(0, 256, 16, dtype=np.uint8)
        b = rng.integers(0, 256, 16, dtype=np.uint8)
        assert (orc.inv_mix_columns(orc.mix_columns(a)) == a).all()
        assert (orc.mix_columns(a ^ b) == (orc.mix_columns(a) ^ orc.mix_columns(b))).all()


def test_mix_columns_unit_columns(orc):
    # M * e_j is column j of circ(2 3 1 1), computed with numpy polynomial arithmetic
    row = _const("mix_row")
    for j in range(4):
        e = np.zeros(16, dtype=np.uint8)
        e[j] = 1
        got = orc.mix_columns(e)[:4]
        want = [row[(j - i) % 4] for i in range(4)]
        assert got.tolist() == want


# ---- key schedule -------------------------------------------------------------------------

def test_rcon_powers(orc):
    p = 1
    for r in range(1, 15):
        assert orc.rcon(r) == p
        p = np_field_mul(p, 2)


def test_appendix_row_schedule_equals_word_rule(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        key = rng.integers(0, 256, 16, dtype=np.uint8)
        a, nra = orc.key_expand(key, 128)
        b, nrb = orc.key_expand_words(key, 4)
        assert nra == nrb == 10 and (a == b).all()
        assert (a[:16] == key).all()


def test_key_sizes(orc):
    for bits, nr in ((128, 10), (192, 12), (256, 14)):
        rk, got = orc.key_expand(np.zeros(bits // 8, dtype=np.uint8), bits)
        assert got == nr and rk.size == 16 * (nr + 1)
    with pytest.raises(ValueError):
        orc.key_expand(np.zeros(20, dtype=np.uint8), 160)


# ---- whole cipher against OpenSSL -----------------------------------------------------------

@pytest.mark.parametrize("key_bits", [128, 192, 256])
def test_ecb_matches_openssl(orc, key_bits):
    rng = np.random.default_rng(key_bits)
    for _ in range(300):
        key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 8, dtype=np.uint8)
        ct = orc.encrypt_blocks(key, data)
        assert ct.tobytes() == openssl_ecb(key.tobytes(), data.tobytes())
        pt = orc.decrypt_blocks(key, ct)
        assert (pt == data).all()
        assert orc.decrypt_blocks(key, data).tobytes() == openssl_ecb(key.tobytes(), data.tobytes(), True)


@pytest.mark.parametrize("key_bits", [128, 256])
def test_one_block_cbc_with_iv_matches_openssl(orc, key_bits):
    # the paper's mode with one block per message: C = E(P ^ IV), P = D(C) ^ IV
    rng = np.random.default_rng(11 + key_bits)
    for _ in range(100):
        key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 4, dtype=np.uint8)
        ct = orc.encrypt_blocks(key, data, iv=iv)
        for j in range(4):
            blk = data[16 * j:16 * j + 16].tobytes()
            assert ct[16 * j:16 * j + 16].tobytes() == openssl_cbc(key.tobytes(), iv.tobytes(), blk)
        assert (orc.decrypt_blocks(key, ct, iv=iv) == data).all()


def test_multiblock_cbc_matches_openssl(orc):
    rng = np.random.default_rng(13)
    for nblk in (1, 2, 5, 33):
        key = rng.integers(0, 256, 16, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * nblk, dtype=np.uint8)
        ct = orc.cbc_encrypt(key, iv, data)
        assert ct.tobytes() == openssl_cbc(key.tobytes(), iv.tobytes(), data.tobytes())
        assert (orc.cbc_decrypt(key, iv, ct) == data).all()


def test_threads_do_not_change_results(orc):
    rng = np.random.default_rng(17)
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    data = rng.integers(0, 256, 16 * 1001, dtype=np.uint8)
    one = orc.encrypt_blocks(key, data, threads=1)
    many = orc.encrypt_blocks(key, data, threads=7)
    assert (one == many).all()


def test_round_trip_random(orc):
    rng = np.random.default_rng(19)
    for bits in (128, 192, 256):
        key = rng.integers(0, 256, bits // 8, dtype=np.uint8)
        iv = rng.integers(0, 256, 16, dtype=np.uint8)
        data = rng.integers(0, 256, 16 * 64, dtype=np.uint8)
        assert (orc.decrypt_blocks(key, orc.encrypt_blocks(key, data, iv=iv), iv=iv) == data).all()


def openssl_ctr(key: bytes, ctr0: bytes, data: bytes) -> bytes:
    c = _openssl()
    op = c.Cipher(c.algorithms.AES(key), c.modes.CTR(ctr0)).encryptor()
    return op.update(data) + op.finalize()


@pytest.mark.parametrize("key_bits", [128, 256])
def test_ctr_matches_openssl_including_counter_wrap(orc, key_bits):
    rng = np.random.default_rng(23 + key_bits)
    for wrap in (False, True):
        key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
        ctr0 = rng.integers(0, 256, 16, dtype=np.uint8)
        if wrap:  # the low 64 bits overflow into the high half, and the whole block wraps
            ctr0[:] = 0xFF
            ctr0[0] = 0x7F
        data = rng.integers(0, 256, 16 * 37, dtype=np.uint8)
        ct = orc.ctr_crypt(key, ctr0, data)
        assert ct.tobytes() == openssl_ctr(key.tobytes(), ctr0.tobytes(), data.tobytes())
        assert (orc.ctr_crypt(key, ctr0, ct) == data).all()
