"""A second, independent structure for the cipher, pinning the oracle: the paper's vectorised
view (Section II) of N messages as an N x 16 byte matrix, where every round step acts on all
rows at once: SubBytes is one table gather over the matrix, ShiftRows a permutation of its 16
columns, MixColumns a 4 x 4 matrix product over GF(2^8) on each group of four columns (here
through a 256 x 256 multiplication table), AddRoundKey an XOR with a broadcast key row.

Nothing here comes from the oracle: the multiplication table is integer polynomial
arithmetic (numpy), the inverse is a table search, the S-box the affine map in its rotation
form, the key schedule the standard word rule, and the round order is the cipher's.  It is
written from those definitions, not from the paper's listing.
"""
import numpy as np
import pytest

from test_oracle_field import np_field_mul


def _mul_table() -> np.ndarray:
    t = np.zeros((256, 256), dtype=np.uint8)
    # multiplication by 2 from the polynomial definition, then the table by linearity
    x2 = np.array([np_field_mul(a, 2) for a in range(256)], dtype=np.uint8)
    t[1] = np.arange(256, dtype=np.uint8)
    for k in range(1, 8):
        t[1 << k] = x2[t[1 << (k - 1)]]
    for c in range(256):
        acc = np.zeros(256, dtype=np.uint8)
        for k in range(8):
            if (c >> k) & 1:
                acc ^= t[1 << k]
        t[c] = acc
    return t


MUL = _mul_table()
INV = np.array([0] + [int(np.nonzero(MUL[a] == 1)[0][0]) for a in range(1, 256)], dtype=np.uint8)


def _rotl(x, s):
    return ((x << s) | (x >> (8 - s))) & 0xFF


SBOX = np.array([int(INV[a]) ^ _rotl(int(INV[a]), 1) ^ _rotl(int(INV[a]), 2) ^ _rotl(int(INV[a]), 3)
                 ^ _rotl(int(INV[a]), 4) ^ 0x63 for a in range(256)], dtype=np.uint8)
INV_SBOX = np.argsort(SBOX).astype(np.uint8)  # the inverse permutation
# ShiftRows on the column-major state (byte i = row i % 4, column i // 4): row r moves left by
# r, so output byte r + 4c gathers input byte r + 4((c + r) mod 4)
SHIFT = np.array([i % 4 + 4 * ((i // 4 + i % 4) % 4) for i in range(16)])
INV_SHIFT = np.argsort(SHIFT)
MIX = np.array([[2, 3, 1, 1], [1, 2, 3, 1], [1, 1, 2, 3], [3, 1, 1, 2]], dtype=np.uint8)
INV_MIX = np.array([[14, 11, 13, 9], [9, 14, 11, 13], [13, 9, 14, 11], [11, 13, 9, 14]], dtype=np.uint8)


def expand(key: np.ndarray) -> np.ndarray:
    nk = key.size // 4
    nr = nk + 6
    w = [key[4 * i:4 * i + 4].copy() for i in range(nk)]
    rc = 1
    for i in range(nk, 4 * (nr + 1)):
        t = w[i - 1].copy()
        if i % nk == 0:
            t = SBOX[np.roll(t, -1)]
            t[0] ^= rc
            rc = int(MUL[rc, 2])
        elif nk > 6 and i % nk == 4:
            t = SBOX[t]
        w.append(w[i - nk] ^ t)
    return np.concatenate(w).reshape(nr + 1, 16)


def mix(state: np.ndarray, m: np.ndarray) -> np.ndarray:
    out = np.zeros_like(state)
    for c in range(4):
        cols = state[:, 4 * c:4 * c + 4]
        for i in range(4):
            acc = np.zeros(state.shape[0], dtype=np.uint8)
            for k in range(4):
                acc ^= MUL[m[i, k], cols[:, k]]
            out[:, 4 * c + i] = acc
    return out


def encrypt_matrix(key, pt):
    rk = expand(key)
    nr = rk.shape[0] - 1
    s = pt ^ rk[0]
    for r in range(1, nr + 1):
        s = SBOX[s][:, SHIFT]
        if r < nr:
            s = mix(s, MIX)
        s = s ^ rk[r]
    return s


def decrypt_matrix(key, ct):
    rk = expand(key)
    nr = rk.shape[0] - 1
    s = ct ^ rk[nr]
    for r in range(nr - 1, -1, -1):
        s = INV_SBOX[s[:, INV_SHIFT]]
        s = s ^ rk[r]
        if r > 0:
            s = mix(s, INV_MIX)
    return s


def test_tables_are_consistent():
    for a in range(1, 256):
        assert MUL[a, INV[a]] == 1
    assert SBOX[0] == 0x63 and sorted(SBOX.tolist()) == list(range(256))
    assert (INV_SBOX[SBOX] == np.arange(256)).all()
    s = np.arange(16)
    assert (s[SHIFT][INV_SHIFT] == s).all()


@pytest.mark.parametrize("key_bytes", [16, 24, 32])
def test_matrix_cipher_matches_oracle(orc, key_bytes):
    rng = np.random.default_rng(300 + key_bytes)
    for _ in range(5):
        key = rng.integers(0, 256, key_bytes, dtype=np.uint8)
        pt = rng.integers(0, 256, (500, 16), dtype=np.uint8)
        ct = encrypt_matrix(key, pt)
        assert (ct.reshape(-1) == orc.encrypt_blocks(key, pt.reshape(-1))).all()
        assert (decrypt_matrix(key, ct) == pt).all()
        assert (decrypt_matrix(key, pt).reshape(-1) == orc.decrypt_blocks(key, pt.reshape(-1))).all()
