#!/usr/bin/env python
"""Generates aes_bitslice_sbox.cuh: Boolean circuits for the AES S-box and inverse S-box on
bitsliced operands (eight 32-bit planes, plane i = bit i of the byte for 32 blocks).

The circuit is derived here from the field definition, the way the paper defines the S-box
(arXiv:1506.08503 App. A2/A5: the GF(2^8) inverse followed by an affine map), using a
tower-field representation to make the inverse cheap in gates:

  GF(2^8) = F2[x]/(x^8+x^4+x^3+x+1)  is isomorphic to  GF(2^4)[y]/(y^2+y+lambda),
  GF(2^4) = F2[z]/(z^4+z+1).

An element a_h*y + a_l has the inverse (a_h*d')*y + (a_h+a_l)*d', where
d = lambda*a_h^2 + a_h*a_l + a_l^2 and d' = d^-1 in GF(2^4) (0 -> 0).  The change of basis
into the tower, the affine map and the change of basis back are 8x8 matrices over GF(2);
the input-side linear functions are merged into one matrix and reduced with Paar's greedy
common-pair heuristic.  The GF(2^4) inverse (four Boolean functions of four variables) is
emitted as LOP3 instructions: each output bit is `d3 ? f1(d0,d1,d2) : f0(d0,d1,d2)`.

The tower parameters (root zeta of z^4+z+1 in GF(2^8), lambda of trace 1, root eta of
y^2+y+lambda) are searched for the smallest total XOR count.  Every generated circuit is
checked against the field definition on all 256 inputs before it is written.

Usage: python gen_bitslice_sbox.py [output.cuh]   (default: next to this script)
"""
from __future__ import annotations

import itertools
import sys
from pathlib import Path

POLY8 = 0x11B
POLY4 = 0x13  # z^4 + z + 1


# ---- field arithmetic ----------------------------------------------------------------------

def mul(a: int, b: int, poly: int, deg: int) -> int:
    p = 0
    while b:
        if b & 1:
            p ^= a
        b >>= 1
        a <<= 1
        if a >> deg & 1:
            a ^= poly
    return p


def mul8(a, b): return mul(a, b, POLY8, 8)
def mul4(a, b): return mul(a, b, POLY4, 4)


def pow8(a, e):
    r = 1
    for _ in range(e):
        r = mul8(r, a)
    return r


def inv8(a): return pow8(a, 254) if a else 0


def inv4(a):
    if not a:
        return 0
    for b in range(1, 16):
        if mul4(a, b) == 1:
            return b
    raise AssertionError


def rotl8(x, s): return ((x << s) | (x >> (8 - s))) & 0xFF


def affine(b): return b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63
def inv_affine(x): return rotl8(x, 1) ^ rotl8(x, 3) ^ rotl8(x, 6) ^ 0x05


def sbox(x): return affine(inv8(x))
def inv_sbox(x): return inv8(inv_affine(x))


# ---- GF(2) matrices as lists of row bitmasks ------------------------------------------------

def mat_from_map(f, nin: int, nout: int) -> list[int]:
    """Rows of the matrix of the GF(2)-linear map f (ints -> ints): row i, bit j = dout_i/din_j."""
    cols = [f(1 << j) for j in range(nin)]
    return [sum(((cols[j] >> i) & 1) << j for j in range(nin)) for i in range(nout)]


def mat_apply(rows: list[int], v: int) -> int:
    return sum((bin(r & v).count("1") & 1) << i for i, r in enumerate(rows))


def mat_inv(rows: list[int], n: int) -> list[int]:
    a = [(rows[i], 1 << i) for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if a[i][0] >> c & 1)
        a[c], a[p] = a[p], a[c]
        for i in range(n):
            if i != c and a[i][0] >> c & 1:
                a[i] = (a[i][0] ^ a[c][0], a[i][1] ^ a[c][1])
    return [a[i][1] for i in range(n)]


# ---- tower ---------------------------------------------------------------------------------

def towers():
    zetas = [z for z in range(256) if pow8(z, 4) ^ z ^ 1 == 0]
    for zeta in zetas:
        emb = lambda a4: _embed(a4, zeta)  # noqa: E731
        for lam in range(16):
            # y^2 + y + lam irreducible over GF(2^4) <=> no root in GF(2^4)
            if any(mul4(t, t) ^ t ^ lam == 0 for t in range(16)):
                continue
            lam8 = emb(lam)
            for eta in range(256):
                if mul8(eta, eta) ^ eta ^ lam8 == 0:
                    yield zeta, lam, eta


def _embed(a4: int, zeta: int) -> int:
    r, p = 0, 1
    for i in range(4):
        if a4 >> i & 1:
            r ^= p
        p = mul8(p, zeta)
    return r


def tower_matrix(zeta: int, eta: int) -> list[int]:
    """T: tower coordinates (low nibble a_l, high nibble a_h) -> polynomial-basis byte."""
    def t(v):
        return _embed(v & 15, zeta) ^ mul8(eta, _embed(v >> 4, zeta))
    return mat_from_map(t, 8, 8)


# ---- Paar's greedy XOR reduction -----------------------------------------------------------

def paar(rows: list[int], nin: int):
    """Returns (ops, outputs): ops is a list of (new_signal, a, b) meaning s_new = s_a ^ s_b;
    outputs[i] is the signal index that holds row i (or -1 for a zero row)."""
    rows = list(rows)
    nsig = nin
    ops = []
    while True:
        best, best_cnt = None, 1
        for a in range(nsig):
            for b in range(a + 1, nsig):
                m = (1 << a) | (1 << b)
                cnt = sum(1 for r in rows if r & m == m)
                if cnt > best_cnt:
                    best, best_cnt = (a, b), cnt
        if best is None:
            break
        a, b = best
        m = (1 << a) | (1 << b)
        ops.append((nsig, a, b))
        rows = [(r & ~m) | (1 << nsig) if r & m == m else r for r in rows]
        nsig += 1
    outs = []
    for r in rows:
        bits = [i for i in range(nsig) if r >> i & 1]
        if not bits:
            outs.append([])
        else:
            outs.append(bits)
    return ops, outs


def xor_count(rows: list[int], nin: int) -> int:
    ops, outs = paar(rows, nin)
    return len(ops) + sum(max(0, len(o) - 1) for o in outs)


# ---- circuit assembly ----------------------------------------------------------------------

class Circuit:
    """Straight-line program over named 32-bit signals, evaluated in Python on 256-bit ints
    (bit x of a signal = value for input byte x) for the exhaustive check, and printed as CUDA."""

    def __init__(self):
        self.lines: list[str] = []
        self.n = 0

    def tmp(self) -> str:
        self.n += 1
        return f"t{self.n}"

    def emit(self, line: str):
        self.lines.append(line)


def gen_linear(c: Circuit, rows: list[int], ins: list[str], consts: int = 0) -> list[str]:
    ops, outs = paar(rows, len(ins))
    sig = list(ins)
    for new, a, b in ops:
        t = c.tmp()
        c.emit(f"const uint32_t {t} = {sig[a]} ^ {sig[b]};")
        sig.append(t)
    res = []
    for i, bits in enumerate(outs):
        t = c.tmp()
        expr = " ^ ".join(sig[b] for b in bits) if bits else "0u"
        if consts >> i & 1:
            expr = f"~({expr})"
        c.emit(f"const uint32_t {t} = {expr};")
        res.append(t)
    return res


def gen_mul4(c: Circuit, a: list[str], b: list[str]) -> list[str]:
    """GF(2^4) product, schoolbook with the reduction z^4 = z + 1 folded in."""
    # coefficient of z^k in the unreduced product: sum over i + j = k of a_i b_j
    terms = {k: [(i, k - i) for i in range(4) if 0 <= k - i < 4] for k in range(7)}
    # reduce: z^4 -> z + 1, z^5 -> z^2 + z, z^6 -> z^3 + z^2
    red = {k: [k] for k in range(4)}
    red[4], red[5], red[6] = [0, 1], [1, 2], [2, 3]
    out_terms = {k: [] for k in range(4)}
    shared = {}
    for k in (4, 5, 6):
        t = c.tmp()
        c.emit(f"const uint32_t {t} = " + " ^ ".join(f"({a[i]} & {b[j]})" for i, j in terms[k]) + ";")
        shared[k] = t
    for k in range(7):
        for o in red[k]:
            out_terms[o].append(shared[k] if k >= 4 else " ^ ".join(f"({a[i]} & {b[j]})" for i, j in terms[k]))
    res = []
    for o in range(4):
        t = c.tmp()
        c.emit(f"const uint32_t {t} = " + " ^ ".join(out_terms[o]) + ";")
        res.append(t)
    return res


def lut(f) -> int:
    """PTX lop3 immediate for f(a, b, c) with a = 0xF0, b = 0xCC, c = 0xAA."""
    v = 0
    for bit in range(8):
        a, b, cc = (0xF0 >> bit) & 1, (0xCC >> bit) & 1, (0xAA >> bit) & 1
        v |= (f(a, b, cc) & 1) << bit
    return v


def gen_inv4(c: Circuit, d: list[str]) -> list[str]:
    res = []
    for bit in range(4):
        def f(hi):
            return lambda x0, x1, x2: (inv4(x0 | x1 << 1 | x2 << 2 | hi << 3) >> bit) & 1
        f0, f1 = c.tmp(), c.tmp()
        c.emit(f"const uint32_t {f0} = lop3<0x{lut(f(0)):02X}>({d[0]}, {d[1]}, {d[2]});")
        c.emit(f"const uint32_t {f1} = lop3<0x{lut(f(1)):02X}>({d[0]}, {d[1]}, {d[2]});")
        t = c.tmp()
        c.emit(f"const uint32_t {t} = lop3<0xCA>({d[3]}, {f1}, {f0});  // d3 ? f1 : f0")
        res.append(t)
    return res


def build_sbox(inverse: bool, zeta: int, lam: int, eta: int) -> tuple[Circuit, int]:
    T = tower_matrix(zeta, eta)
    Ti = mat_inv(T, 8)
    A = mat_from_map(lambda v: affine(v) ^ 0x63, 8, 8)  # linear part of the affine map
    Ai = mat_from_map(lambda v: inv_affine(v) ^ 0x05, 8, 8)
    if inverse:
        # v = Ti * Ai * (x ^ 0x63)  (= Ti*Ai*x ^ Ti*0x05), output = T * w
        lin_in = [mat_apply(Ti, mat_apply(Ai, 1 << j)) for j in range(8)]
        cin = mat_apply(Ti, 0x05)
        out_rows, cout = T, 0
    else:
        lin_in = [mat_apply(Ti, 1 << j) for j in range(8)]
        cin = 0
        out_rows = [sum(((mat_apply(A, mat_apply(T, 1 << j)) >> i) & 1) << j for j in range(8)) for i in range(8)]
        cout = 0x63
    # the 8 tower coordinates v as rows over x
    vrows = [sum(((lin_in[j] >> i) & 1) << j for j in range(8)) for i in range(8)]
    # extra linear signals of the input layer: s = a_h ^ a_l and dlin = lam*a_h^2 ^ a_l^2
    srows = [vrows[i] ^ vrows[4 + i] for i in range(4)]
    sq_l = mat_from_map(lambda a: mul4(lam, mul4(a, a)), 4, 4)
    sq = mat_from_map(lambda a: mul4(a, a), 4, 4)
    drows = []
    for i in range(4):
        r = 0
        for j in range(4):
            if sq_l[i] >> j & 1:
                r ^= vrows[4 + j]
            if sq[i] >> j & 1:
                r ^= vrows[j]
        drows.append(r)
    cs = 0
    cd = 0
    for i in range(4):
        cs |= (((cin >> i) ^ (cin >> (4 + i))) & 1) << i
        cd |= (mat_apply(sq_l, cin >> 4) ^ mat_apply(sq, cin & 15)) >> i << i & (1 << i)
    all_rows = vrows + srows + drows
    consts = cin | (cs << 8) | (cd << 12)
    c = Circuit()
    xs = [f"x{i}" for i in range(8)]
    sig = gen_linear(c, all_rows, xs, consts)
    al, ah, s, dl = sig[0:4], sig[4:8], sig[8:12], sig[12:16]
    prod = gen_mul4(c, ah, al)
    d = []
    for i in range(4):
        t = c.tmp()
        c.emit(f"const uint32_t {t} = {dl[i]} ^ {prod[i]};")
        d.append(t)
    di = gen_inv4(c, d)
    wh = gen_mul4(c, ah, di)
    wl = gen_mul4(c, s, di)
    w = wl + wh
    ys = gen_linear(c, out_rows, w, cout)
    for i in range(8):
        c.emit(f"x{i} = {ys[i]};")
    gates = xor_count(all_rows, 8) + xor_count(out_rows, 8)
    return c, gates


def evaluate(c: Circuit) -> list[int]:
    """Runs the circuit on all 256 inputs at once (signals are 256-bit Python ints)."""
    full = (1 << 256) - 1
    env = {f"x{i}": sum(((x >> i) & 1) << x for x in range(256)) for i in range(8)}

    def lop3(imm, a, b, cc):
        r = 0
        for bit in range(8):
            if imm >> bit & 1:
                ta, tb, tc = (bit >> 2) & 1, (bit >> 1) & 1, bit & 1
                r |= (a if ta else full & ~a) & (b if tb else full & ~b) & (cc if tc else full & ~cc)
        return r

    import re
    for line in c.lines:
        m = re.match(r"(?:const uint32_t )?(\w+) = (.*);", line.split("  //")[0])
        name, expr = m.group(1), m.group(2)
        lm = re.match(r"lop3<0x([0-9A-F]+)>\((\w+), (\w+), (\w+)\)", expr)
        if lm:
            env[name] = lop3(int(lm.group(1), 16), env[lm.group(2)], env[lm.group(3)], env[lm.group(4)])
            continue
        py = expr.replace("0u", "0")
        val = eval(py, {}, env)  # noqa: S307 (expressions we generated ourselves)
        env[name] = val & full
    return [sum(((env[f"x{i}"] >> x) & 1) << i for i in range(8)) for x in range(256)]


def best_tower(inverse: bool):
    best = None
    for zeta, lam, eta in towers():
        c, gates = build_sbox(inverse, zeta, lam, eta)
        if best is None or gates < best[0]:
            best = (gates, zeta, lam, eta, c)
    return best


HEADER = """// aes_bitslice_sbox.cuh -- GENERATED by gen_bitslice_sbox.py; do not edit by hand.
//
// Bitsliced AES S-box and inverse S-box: eight 32-bit planes in place, plane i holds bit i of
// one state byte for 32 blocks.  Derived from the field definition (GF(2^8) inverse followed
// by the affine map of App. A2; the inverse map of App. A5 followed by the inverse) through
// the tower GF((2^4)^2); checked by the generator on all 256 inputs.
//   S-box tower:      zeta = 0x{sz:02X} (root of z^4+z+1), lambda = 0x{sl:X}, eta = 0x{se:02X}; linear-layer XORs = {sg}
//   inverse tower:    zeta = 0x{iz:02X}, lambda = 0x{il:X}, eta = 0x{ie:02X}; linear-layer XORs = {ig}
// Every memory access is absent: the circuit's time does not depend on data or key.
#pragma once
#include <cstdint>

namespace aesgb {{
namespace bs {{

template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {{
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}}

"""


def render(name: str, c: Circuit) -> str:
    args = ", ".join(f"uint32_t& x{i}" for i in range(8))
    body = "\n".join("  " + l for l in c.lines)
    return f"__device__ __forceinline__ void {name}({args}) {{\n{body}\n}}\n\n"


def main():
    out = Path(sys.argv[1]) if len(sys.argv) > 1 else Path(__file__).with_name("aes_bitslice_sbox.cuh")
    fwd = best_tower(False)
    inv = best_tower(True)
    assert evaluate(fwd[4]) == [sbox(x) for x in range(256)], "forward circuit is wrong"
    assert evaluate(inv[4]) == [inv_sbox(x) for x in range(256)], "inverse circuit is wrong"
    text = HEADER.format(sz=fwd[1], sl=fwd[2], se=fwd[3], sg=fwd[0], iz=inv[1], il=inv[2], ie=inv[3], ig=inv[0])
    text += render("sbox_planes", fwd[4]) + render("inv_sbox_planes", inv[4])
    text += "}  // namespace bs\n}  // namespace aesgb\n"
    out.write_text(text)
    print(f"wrote {out}: forward {len(fwd[4].lines)} statements, inverse {len(inv[4].lines)} statements")


if __name__ == "__main__":
    main()
