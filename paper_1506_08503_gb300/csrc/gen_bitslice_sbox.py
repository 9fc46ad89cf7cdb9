#!/usr/bin/env python
"""Generates aes_bitslice_sbox.cuh: the AES S-box and inverse S-box as networks of three-input
logic instructions (LOP3) on bitsliced operands (eight 32-bit planes, plane i = bit i of the
byte for 32 blocks).

The circuit is derived here from the field definition, the way the paper defines the S-box
(arXiv:1506.08503 App. A2/A5: the GF(2^8) inverse followed by an affine map), in three steps.

1. Tower field.  GF(2^8) is written as GF(16)^2, GF(16) as GF(4)^2 and GF(4) as GF(2)^2, each
   over a normal basis, the representation Canright used for compact S-boxes and Boyar and
   Peralta for their low-gate circuits:
     GF(4)  = GF(2)(W),  W^2 + W + 1 = 0,       basis {W, W^2};
     GF(16) = GF(4)(Z),  Z^2 + Z + N = 0,       basis {Z, Z^4},  N in {W, W^2};
     GF(256)= GF(16)(Y), Y^2 + Y + L = 0,       basis {Y, Y^16}, L of trace 1 in GF(16).
   In a normal basis {r, r^q} with r + r^q = 1 and r r^q = c, the inverse of A = a1 r + a0 r^q
   is (a0 e) r + (a1 e) r^q with e = (a1 a0 + c (a1 + a0)^2)^-1, and a product needs three
   products in the subfield (Karatsuba): (a1 b1 + c' p) r + (a0 b0 + c' p) r^q with
   p = (a1 + a0)(b1 + b0) (c' = N in GF(16); in GF(4) the same with c' = 1).  So the whole
   inverse takes 9 AND gates for a1 a0, the GF(16) inverse, and 18 AND gates for a0 e, a1 e.
   The operands of all 27 AND gates of the two outer products are fixed linear forms of the
   input byte: the input (top) linear layer computes them and the linear part of d; an output
   (bottom) linear layer recombines the twelve GF(4) product bits into the output byte and
   applies the change of basis back and the affine map.

2. Linear layers.  Each is a set of XOR targets over its inputs, reduced greedily by
   extracting the pair of signals shared by the most remaining targets (Paar's cancellation-free
   heuristic, ties broken at random over several restarts).

3. Mapping onto LOP3.  The resulting network of two-input gates is covered by three-input
   lookup tables, one LOP3 each: every gate is either materialised or absorbed into a consumer
   whose cut (at most three materialised signals) determines it.  The cover with the fewest
   tables is found exactly by an integer program over all 3-feasible cuts (scipy's MILP
   solver, HiGHS).  Constants (the affine map's 0x63, the inverse map's 0x05) and inversions
   are free: they only change the tables.

The tower parameters, the GF(16) inverse's form (its own tower step, or a direct table per
output bit) and the heuristic's restarts are searched for the fewest LOP3s.  Every emitted
network is checked against the field definition on all 256 inputs before it is written.

Usage: python gen_bitslice_sbox.py [output.cuh]            regenerate from the recorded best trials
       python gen_bitslice_sbox.py --search [output.cuh] [restarts] [jobs]   the full search
"""
from __future__ import annotations

import itertools
import random
import sys
from pathlib import Path

import numpy as np

POLY8 = 0x11B


# ---- the AES field ---------------------------------------------------------------------------

def mul8(a: int, b: int) -> int:
    p = 0
    while b:
        if b & 1:
            p ^= a
        b >>= 1
        a <<= 1
        if a & 0x100:
            a ^= POLY8
    return p


def pow8(a: int, e: int) -> int:
    r = 1
    for _ in range(e):
        r = mul8(r, a)
    return r


def inv8(a: int) -> int:
    return pow8(a, 254) if a else 0


def rotl8(x: int, s: int) -> int:
    return ((x << s) | (x >> (8 - s))) & 0xFF


def affine(b: int) -> int:
    return b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63


def inv_affine(x: int) -> int:
    return rotl8(x, 1) ^ rotl8(x, 3) ^ rotl8(x, 6) ^ 0x05


def sbox(x: int) -> int:
    return affine(inv8(x))


def inv_sbox(x: int) -> int:
    return inv8(inv_affine(x))


# ---- GF(2) matrices (rows as bit masks) ------------------------------------------------------

def mat_from_map(f, nin: int, nout: int) -> list[int]:
    """Rows of the GF(2)-linear map f: row i, bit j = output bit i of f(1 << j)."""
    cols = [f(1 << j) for j in range(nin)]
    return [sum(((cols[j] >> i) & 1) << j for j in range(nin)) for i in range(nout)]


def mat_apply(rows: list[int], v: int) -> int:
    return sum((bin(r & v).count("1") & 1) << i for i, r in enumerate(rows))


def mat_mul(a: list[int], b: list[int], nin: int) -> list[int]:
    """Rows of a o b, where b maps nin bits."""
    return mat_from_map(lambda v: mat_apply(a, mat_apply(b, v)), nin, len(a))


def mat_inv(rows: list[int], n: int) -> list[int]:
    a = [(rows[i], 1 << i) for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if a[i][0] >> c & 1)
        a[c], a[p] = a[p], a[c]
        for i in range(n):
            if i != c and a[i][0] >> c & 1:
                a[i] = (a[i][0] ^ a[c][0], a[i][1] ^ a[c][1])
    return [a[i][1] for i in range(n)]


# ---- the tower in normal bases ---------------------------------------------------------------
# Bit layout of a tower byte: bits 0-3 = A0 (coefficient of Y^16), bits 4-7 = A1 (of Y).  In a
# GF(16) nibble: bits 0-1 = a0 (of Z^4), bits 2-3 = a1 (of Z).  In a GF(4) pair: bit 0 = the
# coefficient of W^2, bit 1 = that of W.

def gf4_mul(x: int, y: int) -> int:
    x1, x0, y1, y0 = x >> 1 & 1, x & 1, y >> 1 & 1, y & 1
    q = (x1 ^ x0) & (y1 ^ y0)
    return ((q ^ (x1 & y1)) << 1) | (q ^ (x0 & y0))


def gf4_scale(n: int, p: int) -> int:
    """n * p in GF(4) for the constant n (linear in p)."""
    return gf4_mul(n, p)


def gf16_mul(a: int, b: int, n: int) -> int:
    a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
    p = gf4_mul(a1 ^ a0, b1 ^ b0)
    np_ = gf4_scale(n, p)
    return ((gf4_mul(a1, b1) ^ np_) << 2) | (gf4_mul(a0, b0) ^ np_)


def gf16_sq(a: int, n: int) -> int:
    return gf16_mul(a, a, n)


def gf16_inv(a: int, n: int) -> int:
    if a == 0:
        return 0
    for b in range(1, 16):
        if gf16_mul(a, b, n) == 0b1111:  # 1 = Z + Z^4, and in GF(4) 1 = W + W^2 (bits 11)
            return b
    raise AssertionError("no inverse")


ONE4, ONE16 = 0b11, 0b1111


def gf256_mul(a: int, b: int, n: int, lam: int) -> int:
    a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
    p = gf16_mul(a1 ^ a0, b1 ^ b0, n)
    lp = gf16_mul(lam, p, n)
    return ((gf16_mul(a1, b1, n) ^ lp) << 4) | (gf16_mul(a0, b0, n) ^ lp)


def towers():
    """Every (N, L, embedding) giving a field isomorphic to the AES field: yields (n, lam, T)
    with T the matrix (rows) mapping tower bytes to AES-field bytes."""
    roots = lambda c: [r for r in range(256) if mul8(r, r) ^ r ^ c == 0]  # noqa: E731
    for w in roots(1):
        w2 = mul8(w, w)
        emb4 = lambda v: (w if v >> 1 & 1 else 0) ^ (w2 if v & 1 else 0)  # noqa: E731
        for n in (0b10, 0b01):  # N = W or W^2
            for z in roots(emb4(n)):
                z4 = pow8(z, 4)
                emb16 = lambda v: mul8(emb4(v >> 2), z) ^ mul8(emb4(v & 3), z4)  # noqa: E731
                for lam in range(16):
                    # trace over GF(2) of lam in GF(16) must be 1 for Y^2 + Y + L to be irreducible
                    t, p = 0, lam
                    for _ in range(4):
                        t ^= p
                        p = gf16_sq(p, n)
                    if t != ONE16:
                        continue
                    for y in roots(emb16(lam)):
                        y16 = pow8(y, 16)
                        emb = lambda v: mul8(emb16(v >> 4), y) ^ mul8(emb16(v & 15), y16)  # noqa: E731
                        T = mat_from_map(emb, 8, 8)
                        yield n, lam, T


def check_tower(n: int, lam: int, T: list[int]) -> None:
    """The tower product agrees with the AES field product under T (exhaustive)."""
    emb = [mat_apply(T, v) for v in range(256)]
    assert sorted(emb) == list(range(256))
    for a in range(256):
        for b in range(0, 256, 7):
            assert emb[gf256_mul(a, b, n, lam)] == mul8(emb[a], emb[b])


# ---- networks of gates on 256-bit truth tables -----------------------------------------------
FULL = (1 << 256) - 1


class Net:
    """A straight-line program: node i has fanins (node ids) and a bitwise function; tt[i] is its
    truth table over the 256 input bytes (bit x = value on byte x)."""

    def __init__(self, nin: int):
        self.fanin: list[tuple[int, ...]] = []
        self.fn: list = []
        self.tt: list[int] = []
        self.kind: list[str] = []
        for i in range(nin):
            self.fanin.append(())
            self.fn.append(None)
            self.kind.append("in")
            self.tt.append(sum(((x >> i) & 1) << x for x in range(256)))
        self._memo = {}

    def _add(self, kind, fanin, fn):
        key = (kind, fanin)
        if key in self._memo:
            return self._memo[key]
        self.fanin.append(fanin)
        self.fn.append(fn)
        self.kind.append(kind)
        self.tt.append(fn(*[self.tt[f] for f in fanin]) & FULL)
        self._memo[key] = len(self.tt) - 1
        return len(self.tt) - 1

    def xor(self, a, b):
        return self._add("xor", tuple(sorted((a, b))), lambda u, v: u ^ v)

    def and_(self, a, b):
        return self._add("and", tuple(sorted((a, b))), lambda u, v: u & v)

    def not_(self, a):
        return self._add("not", (a,), lambda u: ~u)

    def lut(self, table: int, a, b, c):
        """Any function of three signals: table bit (4u + 2v + w) = f(u, v, w)."""
        def f(u, v, w, t=table):
            r = 0
            for k in range(8):
                if t >> k & 1:
                    r |= (u if k & 4 else ~u) & (v if k & 2 else ~v) & (w if k & 1 else ~w)
            return r
        return self._add(f"lut{table}", (a, b, c), f)


def _reach(base: np.ndarray, dim: int) -> np.ndarray:
    """D[v] = the fewest elements of `base` whose XOR is v, for every v in GF(2)^dim
    (breadth-first over the whole space; 99 where unreachable)."""
    size = 1 << dim
    D = np.full(size, 99, dtype=np.int16)
    D[0] = 0
    idx = np.arange(size)
    frontier = np.zeros(size, dtype=bool)
    frontier[0] = True
    k = 0
    while frontier.any():
        k += 1
        nxt = np.zeros(size, dtype=bool)
        for b in base:
            nxt |= frontier[idx ^ int(b)]
        nxt &= D == 99
        D[nxt] = k
        frontier = nxt
    return D


def linear_layer(net: Net, ins: list[int], rows: list[int], consts: int, rng: random.Random) -> list[int]:
    """Nodes computing the XOR targets rows[i] (bit j = include ins[j]), complemented where bit i
    of consts is set.  Boyar and Peralta's shortest-linear-program heuristic: keep the set S of
    signals computed so far and, for every target t, its distance (the fewest elements of S
    whose XOR is t, less one); add the XOR of two elements of S that most lowers the sum of the
    distances (ties: the larger sum of squared distances, then at random), with any target that
    is one XOR away taken at once.  Distances are exact: the space is small enough to search."""
    dim = len(ins)
    S = [1 << j for j in range(dim)]
    node = {1 << j: ins[j] for j in range(dim)}
    want = [r for r in rows]

    def build(v, a, b):
        node[v] = net.xor(node[a], node[b])
        S.append(v)

    while True:
        D = _reach(np.array(S), dim)
        left = [t for t in set(want) if D[t] > 1]
        if not left:
            break
        # a target one XOR away
        quick = None
        for t in left:
            if D[t] == 2:
                for a in S:
                    if D[t ^ a] == 1 and (t ^ a) in node:
                        quick = (t, a, t ^ a)
                        break
            if quick:
                break
        if quick:
            build(*quick)
            continue
        tl = np.array(left)
        best, best_key = None, None
        for i in range(len(S)):
            for j in range(i + 1, len(S)):
                c = S[i] ^ S[j]
                if c in node or c == 0:
                    continue
                nd = np.minimum(D[tl], D[tl ^ c] + 1)
                key = (-int(nd.sum()), int((nd.astype(np.int64) ** 2).sum()), rng.random())
                if best_key is None or key > best_key:
                    best, best_key = (c, S[i], S[j]), key
        build(*best)
    out = []
    for i, r in enumerate(rows):
        if r not in node:
            raise AssertionError("target not built")
        v = node[r]
        if consts >> i & 1:
            v = net.not_(v)
        out.append(v)
    return out


def linear_layer3(net: Net, ins: list[int], rows: list[int], consts: int, rng: random.Random) -> list[int]:
    """As linear_layer, for three-input XORs (one LOP3 each): every new signal is the XOR of two
    or three signals computed so far, chosen to lower most the number of three-input XORs the
    targets still need (a target that is the XOR of m signals needs ceil((m - 1) / 2));
    distances are exact, ties go to the smaller sum of distances, then at random."""
    dim = len(ins)
    S = [1 << j for j in range(dim)]
    node = {1 << j: ins[j] for j in range(dim)}
    want = sorted(set(rows))

    def cost(d):
        return np.maximum(0, (d - 1 + 1) // 2)  # ceil((d - 1) / 2) for d >= 1

    while True:
        D = _reach(np.array(S), dim)
        left = np.array([t for t in want if t not in node])
        if len(left) == 0:
            break
        cur = int(cost(D[left].astype(np.int64)).sum())
        cands = {}
        for i in range(len(S)):
            for j in range(i + 1, len(S)):
                c = S[i] ^ S[j]
                if c and c not in node:
                    cands.setdefault(c, (S[i], S[j]))
                for k in range(j + 1, len(S)):
                    c3 = c ^ S[k]
                    if c3 and c3 not in node and c3 not in cands:
                        cands[c3] = (S[i], S[j], S[k])
        cv = np.array(list(cands.keys()))
        nd = np.minimum(D[left][None, :], D[left[None, :] ^ cv[:, None]] + 1).astype(np.int64)
        gain = cur - cost(nd).sum(axis=1)
        dsum = nd.sum(axis=1)
        order = np.lexsort((np.array([rng.random() for _ in range(len(cv))]), dsum, -gain))
        c = int(cv[order[0]])
        parts = cands[c]
        if len(parts) == 2:
            node[c] = net.xor(node[parts[0]], node[parts[1]])
        else:
            node[c] = net.lut(0x96, node[parts[0]], node[parts[1]], node[parts[2]])
        S.append(c)
    out = []
    for i, r in enumerate(rows):
        v = node[r]
        if consts >> i & 1:
            v = net.not_(v)
        out.append(v)
    return out


# ---- the S-box network ------------------------------------------------------------------------

def forms4(net: Net, x1: int, x0: int) -> tuple[int, int, int]:
    """The three AND operands a GF(4) product needs from one factor: x1, x0, x1 + x0."""
    return (x1, x0, net.xor(x1, x0))


def gf4_mul_net(net: Net, xf, yf) -> tuple[int, int]:
    """(q + x1 y1, q + x0 y0) with q = (x1 + x0)(y1 + y0): the W and W^2 coefficients."""
    q = net.and_(xf[2], yf[2])
    return net.xor(net.and_(xf[0], yf[0]), q), net.xor(net.and_(xf[1], yf[1]), q)


def gf16_products(net: Net, af, bf) -> list[tuple[int, int]]:
    """The three GF(4) products of a GF(16) product (a1 b1, a0 b0, (a1 + a0)(b1 + b0)), each
    as (W, W^2) coefficient nodes; af/bf are the nine forms of each factor."""
    return [gf4_mul_net(net, af[0:3], bf[0:3]), gf4_mul_net(net, af[3:6], bf[3:6]),
            gf4_mul_net(net, af[6:9], bf[6:9])]


def form_rows(coord_rows: list[int]) -> list[int]:
    """The nine AND-operand forms of a GF(16) element from the rows of its four coordinates
    (bit order a0.W^2, a0.W, a1.W^2, a1.W): a1: (W, W^2, sum), a0: (...), a1 + a0: (...)."""
    a0l, a0h, a1l, a1h = coord_rows
    s_l, s_h = a1l ^ a0l, a1h ^ a0h
    return [a1h, a1l, a1h ^ a1l, a0h, a0l, a0h ^ a0l, s_h, s_l, s_h ^ s_l]


def product_to_coords_matrix(n: int) -> list[int]:
    """Rows over the six GF(4) product bits [P11.W, P11.W2, P00.W, P00.W2, Pm.W, Pm.W2] of the
    four coordinates of the GF(16) product: Z coeff = P11 + N Pm, Z^4 coeff = P00 + N Pm."""
    def f(v):
        p11 = (v >> 0 & 1) << 1 | (v >> 1 & 1)
        p00 = (v >> 2 & 1) << 1 | (v >> 3 & 1)
        pm = (v >> 4 & 1) << 1 | (v >> 5 & 1)
        npm = gf4_scale(n, pm)
        return ((p11 ^ npm) << 2) | (p00 ^ npm)
    return mat_from_map(f, 6, 4)


def build(inverse: bool, n: int, lam: int, T: list[int], inv16_mode: str, rng: random.Random,
          lin=None) -> tuple[Net, list[int]]:
    linear = lin or linear_layer
    Ti = mat_inv(T, 8)
    if inverse:
        # x' = Ainv(y) ^ 0x05, v = Ti x'; output = T (inverse in the tower)
        Ai = mat_from_map(lambda v: inv_affine(v) ^ 0x05, 8, 8)
        M_in = mat_mul(Ti, Ai, 8)
        c_in = mat_apply(Ti, 0x05)
        M_out, c_out = T, 0
    else:
        A = mat_from_map(lambda v: affine(v) ^ 0x63, 8, 8)
        M_in, c_in = Ti, 0
        M_out, c_out = mat_mul(A, T, 8), 0x63
    net = Net(8)
    x = list(range(8))
    # tower coordinates of the input as rows over x (with constants)
    v_rows = M_in  # row i = coordinate i
    v_c = c_in
    A0_rows, A1_rows = v_rows[0:4], v_rows[4:8]
    A0_c, A1_c = v_c & 15, v_c >> 4
    f1, f0 = form_rows(A1_rows), form_rows(A0_rows)
    f1c = form_rows([A1_c >> i & 1 for i in range(4)])
    f0c = form_rows([A0_c >> i & 1 for i in range(4)])
    # linear part of d: L (A1 + A0)^2 (GF(16) squaring and scaling are linear over GF(2))
    sqL = mat_from_map(lambda a: gf16_mul(lam, gf16_sq(a, n), n), 4, 4)
    s_rows = [A1_rows[i] ^ A0_rows[i] for i in range(4)]
    g_rows = [sum(s_rows[j] for j in range(4) if False) for _ in range(4)]
    g_rows = []
    for i in range(4):
        r = 0
        for j in range(4):
            if sqL[i] >> j & 1:
                r ^= s_rows[j]
        g_rows.append(r)
    g_c = mat_apply(sqL, A1_c ^ A0_c)
    targets = f1 + f0 + g_rows
    consts = 0
    for i, c in enumerate(f1c + f0c + [g_c >> k & 1 for k in range(4)]):
        consts |= (c & 1) << i
    # drop duplicate/zero targets: map each distinct nonzero row once
    top = linear(net, x, targets, consts, rng)
    F1, F0, G = top[0:9], top[9:18], top[18:22]
    # d = A1 A0 + L (A1 + A0)^2
    P = gf16_products(net, F1, F0)
    pbits = [b for pr in P for b in pr]  # [P11.W, P11.W2, P00.W, P00.W2, Pm.W, Pm.W2]
    Mp = product_to_coords_matrix(n)
    d = linear(net, pbits + G, [Mp[i] | (1 << (6 + i)) for i in range(4)], 0, rng)
    # e = d^-1 in GF(16)
    if inv16_mode == "tower":
        # d = d1 Z + d0 Z^4 over GF(4): f = d1 d0 + N (d1 + d0)^2, f^-1 = f^2 (a swap in the normal
        # basis), e = (d0 f^-1) Z + (d1 f^-1) Z^4
        d0l, d0h, d1l, d1h = d
        df1 = forms4(net, d1h, d1l)
        df0 = forms4(net, d0h, d0l)
        q = gf4_mul_net(net, df1, df0)  # (W, W^2) coefficients of d1 d0
        # N (d1 + d0)^2: squaring swaps the two coordinates; then scale by N
        sh, sl = net.xor(d1h, d0h), net.xor(d1l, d0l)
        sq = (sl, sh)  # (W coeff, W^2 coeff) of (d1 + d0)^2

        def scale(nc, pair):
            hi, lo = pair
            if nc == 0b10:  # W * (p1 W + p0 W^2) = p0 W + (p1 + p0) W^2
                return lo, net.xor(hi, lo)
            return net.xor(hi, lo), hi  # W^2 * (...) = (p1 + p0) W + p1 W^2

        nsq = scale(n, sq)
        fw, fw2 = net.xor(q[0], nsq[0]), net.xor(q[1], nsq[1])
        finv = (fw2, fw)  # squaring swaps
        ff = forms4(net, finv[0], finv[1])
        e1 = gf4_mul_net(net, df0, ff)
        e0 = gf4_mul_net(net, df1, ff)
        e = [e0[1], e0[0], e1[1], e1[0]]  # bits: e0.W2, e0.W, e1.W2, e1.W
    else:
        # each output bit of the GF(16) inverse as a table of four inputs: a multiplexer on one
        # input between two three-input tables (the best variable per bit)
        dtt = [net.tt[b] for b in d]
        e = []
        for bit in range(4):
            def val(dv, b=bit):
                return gf16_inv(dv, n) >> b & 1
            best = None
            for sel in range(4):
                others = [j for j in range(4) if j != sel]
                tabs = []
                for sv in (0, 1):
                    t = 0
                    for k in range(8):
                        dv = sv << sel
                        for pos, j in enumerate(others):
                            dv |= ((k >> (2 - pos)) & 1) << j
                        t |= val(dv) << k
                    tabs.append(t)
                cost = sum(0 if t in (0, 0xFF, 0xF0, 0x0F, 0xCC, 0x33, 0xAA, 0x55) else 1 for t in tabs) + 1
                if best is None or cost < best[0]:
                    best = (cost, sel, others, tabs)
            _, sel, others, tabs = best
            l0 = net.lut(tabs[0], d[others[0]], d[others[1]], d[others[2]])
            l1 = net.lut(tabs[1], d[others[0]], d[others[1]], d[others[2]])
            e.append(net.lut(0xCA, d[sel], l1, l0))  # sel ? l1 : l0  (table bit 4s + 2a + b)
        del dtt
    E = [e[3], e[2], net.xor(e[3], e[2]), e[1], e[0], net.xor(e[1], e[0]),
         net.xor(e[3], e[1]), net.xor(e[2], e[0])]
    E.append(net.xor(E[2], E[5]))
    # inverse = (A0 e) Y + (A1 e) Y^16: tower bits 4-7 from A0 e, bits 0-3 from A1 e
    Q_hi = gf16_products(net, F0, E)  # A0 e
    Q_lo = gf16_products(net, F1, E)  # A1 e
    qbits = [b for pr in Q_lo for b in pr] + [b for pr in Q_hi for b in pr]
    # tower bits of the inverse from the 12 product bits, then M_out
    W = np.zeros((8, 12), dtype=np.uint8)
    for i in range(4):
        for j in range(6):
            W[i, j] = Mp[i] >> j & 1
            W[4 + i, 6 + j] = Mp[i] >> j & 1
    rows = []
    for i in range(8):
        r = 0
        for k in range(8):
            if M_out[i] >> k & 1:
                for j in range(12):
                    if W[k, j]:
                        r ^= 1 << j
        rows.append(r)
    outs = linear(net, qbits, rows, c_out, rng)
    return net, outs


# ---- exact cover by three-input tables ---------------------------------------------------------

def cuts(net: Net, k: int = 3) -> list[list[frozenset]]:
    cs: list[list[frozenset]] = []
    for v in range(len(net.tt)):
        if net.kind[v] == "in":
            cs.append([frozenset([v])])
            continue
        acc = {frozenset([v])}
        parts = [cs[f] for f in net.fanin[v]]
        for combo in itertools.product(*parts):
            u = frozenset().union(*combo)
            if len(u) <= k:
                acc.add(u)
        cs.append(sorted(acc, key=lambda c: (len(c), sorted(c))))
    return cs


def cone_table(net: Net, v: int, leaves: tuple[int, ...]) -> int:
    """Truth table (8 bits, leaves as u = 0xF0, v = 0xCC, w = 0xAA) of node v over its cut."""
    pats = [0xF0, 0xCC, 0xAA]
    val = {l: pats[i] for i, l in enumerate(leaves)}

    def ev(u):
        if u in val:
            return val[u]
        r = net.fn[u](*[ev(f) for f in net.fanin[u]]) & 0xFF
        val[u] = r
        return r
    return ev(v)


def map_lop3(net: Net, outs: list[int]):
    """Minimum cover of the network by 3-input tables; returns (count, program) where program
    is a list of (node, leaves, table) in topological order."""
    from scipy.optimize import Bounds, LinearConstraint, milp
    from scipy.sparse import lil_matrix

    cs = cuts(net)
    gates = [v for v in range(len(net.tt)) if net.kind[v] != "in"]
    # variables: x_v (materialised) for gates, y_(v, c) for each non-trivial cut of each gate
    xi = {v: i for i, v in enumerate(gates)}
    ycuts = []
    for v in gates:
        for c in cs[v]:
            if c != frozenset([v]):
                ycuts.append((v, c))
    nx, ny = len(gates), len(ycuts)
    nvar = nx + ny
    rows_eq, rows_le = [], []
    # sum_c y_(v,c) - x_v = 0
    by_v = {}
    for j, (v, c) in enumerate(ycuts):
        by_v.setdefault(v, []).append(j)
    A = lil_matrix((nx + sum(len(c) for _, c in ycuts) + len(outs), nvar))
    lo, hi = [], []
    r = 0
    for v in gates:
        for j in by_v.get(v, []):
            A[r, nx + j] = 1
        A[r, xi[v]] = -1
        lo.append(0)
        hi.append(0)
        r += 1
    for j, (v, c) in enumerate(ycuts):
        for u in c:
            if net.kind[u] != "in":
                A[r, nx + j] = 1
                A[r, xi[u]] = -1
                lo.append(-np.inf)
                hi.append(0)
                r += 1
    for o in outs:
        if net.kind[o] != "in":
            A[r, xi[o]] = 1
            lo.append(1)
            hi.append(1)
            r += 1
    A = A[:r].tocsr()
    cost = np.concatenate([np.ones(nx), np.zeros(ny)])
    res = milp(cost, constraints=LinearConstraint(A, lo, hi), integrality=np.ones(nvar), bounds=Bounds(0, 1),
               options={"time_limit": 30})
    if res.x is None:
        raise RuntimeError("cover not found")
    xs = res.x
    chosen = {}
    for j, (v, c) in enumerate(ycuts):
        if xs[nx + j] > 0.5 and xs[xi[v]] > 0.5:
            chosen[v] = tuple(sorted(c))
    prog = []
    for v in gates:
        if xs[xi[v]] > 0.5:
            leaves = chosen[v]
            prog.append((v, leaves, cone_table(net, v, leaves)))
    return len(prog), prog


def evaluate_program(prog, outs: list[int]) -> list[int]:
    """Runs the LOP3 program on all 256 inputs (independent of the network's own tables)."""
    val = {i: sum(((x >> i) & 1) << x for x in range(256)) for i in range(8)}
    for v, leaves, t in prog:
        ins = [val[l] for l in leaves] + [0] * (3 - len(leaves))
        u, w, z = ins
        r = 0
        for k in range(8):
            if t >> k & 1:
                a = u if (0xF0 >> k) & 1 else ~u
                b = w if (0xCC >> k) & 1 else ~w
                c = z if (0xAA >> k) & 1 else ~z
                r |= a & b & c
        val[v] = r & FULL
    return [sum(((val[outs[i]] >> x) & 1) << i for i in range(8)) for x in range(256)]


def lop3_imm(t: int, nleaves: int) -> int:
    """PTX lop3's immediate for table t over (a, b, c) = the leaves (a = 0xF0, b = 0xCC,
    c = 0xAA).  A table over fewer than three leaves does not depend on the unused operand
    positions (cone_table never reads them), so it serves as the immediate whatever is passed
    there."""
    del nleaves
    return t


def table_expressions() -> dict[int, str]:
    """The shortest C expression (fewest operators among ~, &, |, ^) of each of the 256 functions
    of three operands a, b, c, as a table over a = 0xF0, b = 0xCC, c = 0xAA.  The kernel source
    states each table as such an expression; ptxas folds every one into a single LOP3."""
    best = {0xF0: "a", 0xCC: "b", 0xAA: "c", 0x00: "0u", 0xFF: "~0u"}
    cost = {t: 0 for t in best}
    frontier = dict(best)
    for size in range(1, 12):
        found = {}
        items = list(best.items())
        for t, e in items:  # unary
            if cost[t] == size - 1:
                u = ~t & 0xFF
                if u not in best and u not in found:
                    found[u] = f"~{e}" if len(e) <= 2 else f"~({e})"
        for (t1, e1), (t2, e2) in itertools.combinations_with_replacement(items, 2):
            if cost[t1] + cost[t2] + 1 != size:
                continue
            for op, f in (("&", t1 & t2), ("|", t1 | t2), ("^", t1 ^ t2)):
                if f not in best and f not in found:
                    found[f] = f"({e1} {op} {e2})"
        for f, e in found.items():
            best[f] = e
            cost[f] = size
        if len(best) == 256:
            break
    assert len(best) == 256
    return best


_EXPR = None


def c_expr(t: int, ops: list[str]) -> str:
    global _EXPR
    if _EXPR is None:
        _EXPR = table_expressions()
    e = _EXPR[t]
    if e.startswith("(") and e.endswith(")"):
        e = e[1:-1]
    import re
    return re.sub(r"\b([abc])\b", lambda m: ops["abc".index(m.group(1))], e)


def _trial(args):
    inverse, ti, mode, seed = args
    n, lam, T = list(towers())[ti]
    net, outs = build(inverse, n, lam, T, mode, random.Random(seed))
    want = [inv_sbox(x) if inverse else sbox(x) for x in range(256)]
    got = [sum(((net.tt[outs[i]] >> x) & 1) << i for i in range(8)) for x in range(256)]
    assert got == want, "network differs from the field definition"
    gates2 = sum(1 for k in net.kind if k != "in")
    count, prog = map_lop3(net, outs)
    return count, gates2, n, lam, ti, mode, prog, outs, args


def search(inverse: bool, restarts: int, seed: int, jobs: int):
    """Every tower, both forms of the GF(16) inverse, `restarts` tie-breaking seeds each, in
    `jobs` processes; returns the trial with the fewest LOP3s (the first found on ties)."""
    import multiprocessing as mp

    ntow = len(list(towers()))
    tasks = [(inverse, ti, mode, seed * 1_000_003 + 97 * ti + 7 * r + (mode == "table"))
             for ti in range(ntow) for mode in ("tower", "table") for r in range(restarts)]
    best = None
    with mp.get_context("spawn").Pool(jobs) as pool:
        for res in pool.imap(_trial, tasks, chunksize=1):
            if best is None or res[0] < best[0]:
                best = res
                print(f"  {'inverse' if inverse else 'forward'}: {res[0]} LOP3 ({res[1]} two-input gates), "
                      f"tower {res[4]}, N={res[2]:02b} L={res[3]:X} inv16={res[5]}", file=sys.stderr, flush=True)
    return best


HEADER = """// aes_bitslice_sbox.cuh -- GENERATED by gen_bitslice_sbox.py; do not edit by hand.
//
// Bitsliced AES S-box and inverse S-box: eight 32-bit planes in place, plane i holds bit i of
// one state byte for 32 blocks.  Derived from the field definition (GF(2^8) inverse followed
// by the affine map of App. A2; the inverse map of App. A5 followed by the inverse) through a
// normal-basis tower GF(((2^2)^2)^2) with 27 AND gates in the two outer products, mapped onto
// three-input LOP3 instructions by an exact cover; checked by the generator on all 256 inputs.
//   S-box:          {fc} LOP3 ({fg} two-input gates before mapping), N = {fn}, L = 0x{fl:X}, GF(16) inverse as {fm} (tower {ft[1]}, seed {ft[3]})
//   inverse S-box:  {ic} LOP3 ({ig} two-input gates before mapping), N = {inn}, L = 0x{il:X}, GF(16) inverse as {im} (tower {it[1]}, seed {it[3]})
// No memory access, no branch: the circuit's time does not depend on data or key.
// Each statement is one three-input table AES_SBOX_T(immediate, a, b, c, expression): on the
// device one lop3 instruction with the table as its immediate, on the host (the CPU test of
// the rounds) the same table as a C expression.  Left as C expressions on the device, the
// compiler regrouped the tables inside the rolled round loop (84-87 instructions per S-box).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define AES_SBOX_FN __host__ __device__ __forceinline__
#else
#define AES_SBOX_FN inline
#endif
#if defined(__CUDA_ARCH__)
template <uint32_t L>
__device__ __forceinline__ uint32_t aes_lop3(uint32_t a, uint32_t b, uint32_t c) {{
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(L));
  return d;
}}
#define AES_SBOX_T(L, a, b, c, e) aes_lop3<L>(a, b, c)
#else
#define AES_SBOX_T(L, a, b, c, e) (e)
#endif

namespace aesgb {{
namespace bs {{

"""


def allocate(prog, outs: list[int]) -> tuple[dict, int]:
    """Registers for the device block's temporaries by a linear scan over the straight-line
    program: a temporary's register is free again after its last use (outputs stay live to the
    end).  Returns (node -> register index, number of registers)."""
    last = {}
    for k, (v, leaves, t) in enumerate(prog):
        for l in leaves:
            last[l] = k
    for o in outs:
        last[o] = len(prog)
    free, reg, nregs = [], {}, 0
    for k, (v, leaves, t) in enumerate(prog):
        # operands are read before the result is written, so a register freed here can be reused
        for l in set(leaves):
            if l in reg and last[l] == k:
                free.append(reg[l])
        if free:
            reg[v] = free.pop()
        else:
            reg[v] = nregs
            nregs += 1
    return reg, nregs


def render(name: str, prog, outs: list[int]) -> str:
    """The network as one function: each table is AES_SBOX_T(immediate, a, b, c, expression),
    one lop3 on the device (a statement of its own, so that ptxas schedules the tables freely
    but cannot regroup them) and the C expression of the same table on the host.  Tables of
    fewer than three leaves repeat the first leaf in the unused positions (the immediate does
    not depend on them)."""
    args = ", ".join(f"uint32_t& x{i}" for i in range(8))
    nm = {i: f"i{i}" for i in range(8)}
    lines = [f"  const uint32_t i{i} = x{i};" for i in range(8)]
    for v, leaves, t in prog:
        nm[v] = f"t{v}"
        ops = [nm[l] for l in leaves]
        ops += [ops[0]] * (3 - len(ops))
        imm = lop3_imm(t, len(leaves))
        lines.append(f"  const uint32_t t{v} = AES_SBOX_T(0x{imm:02X}, {ops[0]}, {ops[1]}, {ops[2]}, {c_expr(imm, ops)});")
    for i, o in enumerate(outs):
        lines.append(f"  x{i} = {nm[o]};")
    return f"AES_SBOX_FN void {name}({args}) {{\n" + "\n".join(lines) + "\n}\n\n"


# The trials the full search (--search, about 40 minutes on 8 cores) found best, as (inverse,
# tower index, GF(16) inverse form, seed): regenerating from them takes seconds.
BEST = {False: (False, 104, "table", 1 * 1_000_003 + 97 * 104 + 7 * 0 + 1),
        True: (True, 14, "table", 2 * 1_000_003 + 97 * 14 + 7 * 0 + 1)}


def main():
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    out = Path(args[0]) if args else Path(__file__).with_name("aes_bitslice_sbox.cuh")
    for n0, l0, T0 in towers():
        check_tower(n0, l0, T0)
    if "--search" in sys.argv:
        restarts = int(args[1]) if len(args) > 1 else 2
        jobs = int(args[2]) if len(args) > 2 else 8
        fwd = search(False, restarts, 1, jobs)
        inv = search(True, restarts, 2, jobs)
    else:
        fwd, inv = _trial(BEST[False]), _trial(BEST[True])
    for which, b, ref in (("forward", fwd, sbox), ("inverse", inv, inv_sbox)):
        got = evaluate_program(b[6], b[7])
        assert got == [ref(x) for x in range(256)], f"{which} LOP3 program is wrong"
    bn = lambda n: "W" if n == 0b10 else "W^2"  # noqa: E731
    text = HEADER.format(fc=fwd[0], fg=fwd[1], fn=bn(fwd[2]), fl=fwd[3], fm=fwd[5], ft=fwd[8],
                         ic=inv[0], ig=inv[1], inn=bn(inv[2]), il=inv[3], im=inv[5], it=inv[8])
    text += render("sbox_planes", fwd[6], fwd[7]) + render("inv_sbox_planes", inv[6], inv[7])
    text += "}  // namespace bs\n}  // namespace aesgb\n"
    out.write_text(text)
    print(f"wrote {out}: forward {fwd[0]} LOP3, inverse {inv[0]} LOP3")


if __name__ == "__main__":
    main()
