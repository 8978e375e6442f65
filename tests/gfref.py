"""Independent GF(2^w) arithmetic used to pin the oracle.

Written without tables: multiplication is shift-and-add (carry-less product
reduced bit by bit by the primitive polynomial), the textbook definition of
the field GF(2)[x]/(p(x)).  The oracle uses exp/log tables instead, so a
mistake in either formulation shows up as a disagreement.
"""
from __future__ import annotations

import numpy as np

PRIM = {4: 0x13, 8: 0x11D, 16: 0x1100B}


def mul(a: int, b: int, w: int) -> int:
    p = PRIM[w]
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> w:
            a ^= p
    return r


def mul_np(a, b, w: int) -> np.ndarray:
    """Vectorised shift-and-add product of two uint32 arrays."""
    p = np.uint32(PRIM[w])
    top = np.uint32(1 << w)
    a = np.array(a, dtype=np.uint32, copy=True)
    b = np.array(b, dtype=np.uint32, copy=True)
    a, b = np.broadcast_arrays(a, b)
    a = a.copy(); b = b.copy()
    r = np.zeros(a.shape, dtype=np.uint32)
    for _ in range(w):
        r ^= np.where(b & 1, a, 0).astype(np.uint32)
        b >>= np.uint32(1)
        a <<= np.uint32(1)
        a ^= np.where(a & top, p, 0).astype(np.uint32)
    return r


def power(a: int, e: int, w: int) -> int:
    r = 1
    for _ in range(e):
        r = mul(r, a, w)
    return r


def inv(a: int, w: int) -> int:
    """a^(2^w - 2) by square-and-multiply (Fermat), no tables."""
    if a == 0:
        raise ZeroDivisionError
    e = (1 << w) - 2
    r, base = 1, a
    while e:
        if e & 1:
            r = mul(r, base, w)
        base = mul(base, base, w)
        e >>= 1
    return r


def poly_eval(coeffs, x: int, w: int) -> int:
    """sum_i coeffs[i] x^i by Horner's rule."""
    r = 0
    for c in reversed(list(coeffs)):
        r = mul(r, x, w) ^ int(c)
    return r


def lagrange_eval(xs, ys, x: int, w: int) -> int:
    """Value at x of the unique polynomial of degree < len(xs) through (xs, ys)."""
    total = 0
    for i, (xi, yi) in enumerate(zip(xs, ys)):
        num, den = 1, 1
        for j, xj in enumerate(xs):
            if j != i:
                num = mul(num, x ^ xj, w)
                den = mul(den, xi ^ xj, w)
        total ^= mul(int(yi), mul(num, inv(den, w), w), w)
    return total


def rank(A, w: int) -> int:
    """Rank over GF(2^w) by row reduction."""
    A = [list(map(int, row)) for row in A]
    rows, cols = len(A), len(A[0]) if A else 0
    r = 0
    for c in range(cols):
        piv = next((i for i in range(r, rows) if A[i][c]), None)
        if piv is None:
            continue
        A[r], A[piv] = A[piv], A[r]
        iv = inv(A[r][c], w)
        A[r] = [mul(v, iv, w) for v in A[r]]
        for i in range(rows):
            if i != r and A[i][c]:
                f = A[i][c]
                A[i] = [vi ^ mul(f, vr, w) for vi, vr in zip(A[i], A[r])]
        r += 1
    return r


def symbols(block: np.ndarray, w: int) -> np.ndarray:
    """Symbols of one block: bytes for w <= 8, little-endian uint16 for w = 16."""
    if w == 16:
        return block.view("<u2").astype(np.uint32)
    return block.astype(np.uint32)


def packets_to_symbols(block: np.ndarray, w: int, P: int) -> np.ndarray:
    """Read a packet-layout block as symbols: bit b of packet c in a
    super-packet is bit c of symbol b of that super-packet."""
    nsp = block.size // (w * P)
    out = np.zeros(nsp * P * 8, dtype=np.uint32)
    for sp in range(nsp):
        base = sp * w * P
        for c in range(w):
            pk = block[base + c * P: base + (c + 1) * P]
            bits = np.unpackbits(pk, bitorder="little").astype(np.uint32)
            out[sp * P * 8:(sp + 1) * P * 8] |= bits << np.uint32(c)
    return out
