"""Pins for the oracle's GF(2^8) arithmetic (paper Section II).

Independent references used here:
  * the paper's two worked examples (tests/golden/paper_gf_examples.txt);
  * integer polynomial arithmetic from numpy (np.polymul / np.polydiv over Z, reduced mod 2
    afterwards: division by a monic polynomial commutes with reduction mod 2), which is a
    different computation from the oracle's shift-and-XOR loop;
  * field axioms checked exhaustively or on large samples.
"""
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).parent / "golden" / "paper_gf_examples.txt"
MODULUS = [1, 0, 0, 0, 1, 1, 0, 1, 1]  # x^8 + x^4 + x^3 + x + 1, highest power first (Section II)


def _coeffs(a: int) -> np.ndarray:
    return np.array([(a >> (7 - i)) & 1 for i in range(8)], dtype=np.int64)


def np_field_mul(a: int, b: int) -> int:
    prod = np.polymul(_coeffs(a), _coeffs(b))
    _, rem = np.polydiv(prod.astype(float), np.array(MODULUS, dtype=float))
    rem = np.rint(rem).astype(np.int64) % 2
    return int("".join(str(int(c)) for c in rem), 2) if rem.size else 0


def test_paper_worked_examples(orc):
    lines = [l.split() for l in GOLDEN.read_text().splitlines() if l.strip() and not l.startswith("#")]
    assert len(lines) == 2
    for op, a, b, r in lines:
        a, b, r = int(a, 16), int(b, 16), int(r, 16)
        got = orc.gf_add(a, b) if op == "add" else orc.gf_mul(a, b)
        assert got == r, (op, a, b, got, r)


def test_mul_matches_integer_polynomial_arithmetic_all_pairs(orc):
    # the numpy reference is slow; check every a against a spread of b, and every pair for
    # multiplication by the basis elements x^k, which with distributivity fixes the product
    for a in range(256):
        for k in range(8):
            assert orc.gf_mul(a, 1 << k) == np_field_mul(a, 1 << k)
    rng = np.random.default_rng(0)
    for a, b in rng.integers(0, 256, size=(3000, 2)):
        assert orc.gf_mul(int(a), int(b)) == np_field_mul(int(a), int(b))


def test_mul_field_axioms_exhaustive(orc):
    tab = np.array([[orc.gf_mul(a, b) for b in range(256)] for a in range(256)], dtype=np.int64)
    assert (tab == tab.T).all()                     # commutative
    assert (tab[1] == np.arange(256)).all()         # 1 is the identity
    assert (tab[0] == 0).all()
    # distributive over XOR: a(b + c) = ab + ac, all a, b and a sample of c
    for c in (1, 2, 3, 0x53, 0xCA, 0xFF):
        b = np.arange(256)
        assert (tab[:, b ^ c] == (tab[:, b] ^ tab[:, c][:, None])).all()
    # associative on a sample
    rng = np.random.default_rng(1)
    for a, b, c in rng.integers(0, 256, size=(5000, 3)):
        assert tab[tab[a, b], c] == tab[a, tab[b, c]]
    # no zero divisors: every row of a nonzero a is a permutation (a field)
    for a in range(1, 256):
        assert len(set(tab[a].tolist())) == 256


def test_inverse(orc):
    assert orc.gf_inv(0) == 0  # App. A2 leaves the entry for 0 at 0
    for a in range(1, 256):
        assert orc.gf_mul(a, orc.gf_inv(a)) == 1


def test_generator_order(orc):
    # x + 1 = 0x03 generates the multiplicative group of this field (order 255)
    seen, p = set(), 1
    for _ in range(255):
        seen.add(p)
        p = orc.gf_mul(p, 3)
    assert p == 1 and len(seen) == 255


def test_add_is_xor(orc):
    for a in range(0, 256, 7):
        for b in range(0, 256, 5):
            assert orc.gf_add(a, b) == a ^ b
