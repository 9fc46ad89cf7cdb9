"""Pins for the oracle's S-box and inverse S-box (paper App. A2 and A5).

The oracle builds the S-box as A * inv(x) + b with A the circulant matrix of App. A2 on
MSB-first bit vectors, and the inverse S-box separately as inv(A' x + b') (App. A5).  The
tests pin this against: the rotation form of the same affine map (a different formula:
b ^ rotl(b,1) ^ ... ^ rotl(b,4) ^ 0x63), the values the appendix fixes (S(0) = b,
InvS(0x63) = 0), InvS o S = id, and the cryptographic properties of an inversion-based
S-box that any slip in the inversion or the affine map would destroy (bijectivity, no fixed
or opposite-fixed points, differential uniformity 4, nonlinearity 112).
"""
from pathlib import Path

import numpy as np

CONST = Path(__file__).parent / "golden" / "paper_constants.txt"


def _const(name):
    for line in CONST.read_text().splitlines():
        if line.startswith(name + " "):
            return [int(v) for v in line.split()[1:]]
    raise KeyError(name)


def rotl8(x, s):
    return ((x << s) | (x >> (8 - s))) & 0xFF


def test_affine_rotation_form(orc):
    for b in range(256):
        want = b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63
        assert orc.affine(b) == want


def test_inv_affine_undoes_affine(orc):
    for x in range(256):
        assert orc.inv_affine(orc.affine(x)) == x
        assert orc.affine(orc.inv_affine(x)) == x


def test_appendix_fixed_values(orc):
    b = int("".join(map(str, _const("sbox_b"))), 2)
    assert b == 0x63
    assert orc.sbox(0) == b                          # inv(0) = 0, so S(0) = b (App. A2)
    assert orc.inv_sbox(0x63) == _const("inv_sbox_at_0x63")[0]  # App. A5 sets this entry to 0
    bi = int("".join(map(str, _const("inv_sbox_b"))), 2)
    assert bi == 0x05 and orc.inv_affine(0) == 0x05


def test_sbox_is_affine_of_inverse(orc):
    for x in range(256):
        assert orc.sbox(x) == orc.affine(orc.gf_inv(x))


def test_bijection_and_inverse(orc):
    s = orc.sbox_table()
    si = orc.inv_sbox_table()
    assert len(set(s.tolist())) == 256
    assert (si[s] == np.arange(256)).all()
    assert (s[si] == np.arange(256)).all()


def test_no_fixed_points(orc):
    s = orc.sbox_table().astype(int)
    x = np.arange(256)
    assert not (s == x).any()
    assert not (s == (x ^ 0xFF)).any()


def test_differential_uniformity_and_nonlinearity(orc):
    s = orc.sbox_table().astype(np.int64)
    x = np.arange(256)
    # difference distribution table: max count over nonzero input differences is 4
    ddt_max = 0
    for d in range(1, 256):
        counts = np.bincount(s[x] ^ s[x ^ d], minlength=256)
        ddt_max = max(ddt_max, counts.max())
    assert ddt_max == 4
    # nonlinearity 112: the largest Walsh coefficient over nonzero output masks is 32
    bits = ((x[:, None] >> np.arange(8)) & 1)
    walsh_max = 0
    for b in range(1, 256):
        f = np.bitwise_xor.reduce(((s[:, None] >> np.arange(8)) & 1) & ((b >> np.arange(8)) & 1), axis=1)
        for a in range(256):
            lin = np.bitwise_xor.reduce(bits & ((a >> np.arange(8)) & 1), axis=1)
            walsh_max = max(walsh_max, abs(int(np.sum(1 - 2 * (f ^ lin)))))
    assert 128 - walsh_max // 2 == 112
