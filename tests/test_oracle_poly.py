"""Pins of the oracle's polynomial realization (§3).

Pins: the paper's worked example (§3.1-§3.3), the roots of g(x) and of every
codeword (a codeword is a multiple of g, §3.3), linearity (§3.2's remark on
updates), the encode/decode symmetry (§3.3's first remark), and a
brute-force round trip over every erasure pattern in GF(2^4).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests import gfref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example_rs_4_3_gf256.txt")


def read_golden(path=GOLDEN):
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, vals = line.split(":", 1)
            out[key.strip()] = [int(v) for v in vals.split()]
    return out


def pos(k, m, b):
    return m + b if b < k else b - k


# ------------------------------------------------------------ worked example
def test_worked_example_generator_polynomial():
    g = read_golden()
    assert O.genpoly(8, 3).tolist() == g["genpoly"]


def test_worked_example_encode():
    g = read_golden()
    assert O.poly_encode_column(8, 4, 3, g["data"]).tolist() == g["parity"]


def test_worked_example_decode_steps():
    g = read_golden()
    k, m = 4, 3
    col = g["data"] + g["parity"]
    er = g["erased_blocks"]
    c = list(col)
    for b in er:
        c[b] = 0
    filled, D, V = O.poly_decode_column(8, k, m, er, c)
    assert D.tolist() == g["syndromes"]
    assert V.tolist() == [g["vmatrix_row0"], g["vmatrix_row1"], g["vmatrix_row2"]]
    assert [int(filled[b]) for b in er] == g["solution"]
    assert filled.tolist() == col


def test_worked_example_block_path_matches_column_path():
    g = read_golden()
    blocks = np.zeros((7, 3), dtype=np.uint8)
    for i, v in enumerate(g["data"]):
        blocks[i, :] = v
    O.poly_encode(8, 4, 3, blocks)
    assert blocks[4:, 0].tolist() == g["parity"]
    blocks[0:3, :] = 0
    O.poly_decode(8, 4, 3, g["erased_blocks"], blocks)
    assert blocks[0:3, 2].tolist() == g["solution"]


# ------------------------------------------------------------------ roots
@pytest.mark.parametrize("w,m", [(8, 1), (8, 2), (8, 3), (8, 4), (8, 6), (16, 4), (16, 3), (4, 5)])
def test_generator_roots_are_consecutive_alpha_powers(w, m):
    g = O.genpoly(w, m).tolist()
    assert len(g) == m + 1 and g[-1] == 1
    a = 1
    for i in range(m):
        assert gfref.poly_eval(g, a, w) == 0, (w, m, i)
        a = gfref.mul(a, 2, w)
    # alpha^m is not a root (degree-m polynomial with exactly these m roots)
    assert gfref.poly_eval(g, a, w) != 0


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (16, 12, 4), (8, 20, 4)])
def test_every_codeword_has_the_roots(w, k, m):
    sb = 2 if w == 16 else 1
    B = 24 * sb
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(inputs.stream_seed(1), 3, k, B)
    O.poly_encode(w, k, m, blocks)
    syms = np.stack([gfref.symbols(blocks[b], w) for b in range(k + m)])
    for t in range(syms.shape[1]):
        coeffs = [0] * (k + m)
        for b in range(k + m):
            coeffs[pos(k, m, b)] = int(syms[b, t])
        a = 1
        for j in range(m):
            assert gfref.poly_eval(coeffs, a, w) == 0
            a = gfref.mul(a, 2, w)


def test_parity_is_remainder_by_independent_long_division():
    """Eq. 1 with a table-free division in the test."""
    w, k, m = 8, 10, 4
    d = inputs.random_bytes(99, 0, k).astype(int).tolist()
    g = [1]
    a = 1
    for _ in range(m):  # multiply (x + a) in, g stored highest degree last
        ng = [0] * (len(g) + 1)
        for i, c in enumerate(g):
            ng[i + 1] ^= c
            ng[i] ^= gfref.mul(c, a, w)
        g = ng
        a = gfref.mul(a, 2, w)
    num = [0] * m + d
    for deg in range(len(num) - 1, m - 1, -1):
        lead = num[deg]
        for t in range(m + 1):
            num[deg - m + t] ^= gfref.mul(lead, g[t], w)
    assert O.poly_encode_column(w, k, m, d).tolist() == num[:m]


# --------------------------------------------------------- linearity (§3.2)
@pytest.mark.parametrize("w", [8, 16])
def test_encode_is_linear(w):
    k, m, B = 10, 4, 64
    a = np.zeros((k + m, B), dtype=np.uint8)
    b = np.zeros((k + m, B), dtype=np.uint8)
    a[:k] = inputs.stripe_blocks(11, 0, k, B)
    b[:k] = inputs.stripe_blocks(12, 0, k, B)
    s = np.zeros_like(a)
    s[:k] = a[:k] ^ b[:k]
    O.poly_encode(w, k, m, a)
    O.poly_encode(w, k, m, b)
    O.poly_encode(w, k, m, s)
    assert np.array_equal(s[k:], a[k:] ^ b[k:])


# ----------------------------------------------------------- symmetry (§3.3)
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (16, 12, 4), (8, 6, 3)])
def test_encode_equals_decode_of_erased_parity(w, k, m):
    B = 32
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(5, 1, k, B)
    enc = blocks.copy()
    O.poly_encode(w, k, m, enc)
    dec = blocks.copy()
    dec[k:] = 0xAB  # garbage in the erased slots must not matter
    O.poly_decode(w, k, m, list(range(k, k + m)), dec)
    assert np.array_equal(enc, dec)


# ------------------------------------------------------ round trips at w=8/16
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (16, 12, 4), (8, 6, 3)])
def test_decode_round_trip_seeded_patterns(w, k, m):
    n = k + m
    B = 40
    seed = inputs.stream_seed(1)
    for stripe in range(12):
        blocks = np.zeros((n, B), dtype=np.uint8)
        blocks[:k] = inputs.stripe_blocks(seed, stripe, k, B)
        O.poly_encode(w, k, m, blocks)
        ref = blocks.copy()
        e = 1 + stripe % m
        er = inputs.erasure_pattern(seed, stripe, n, e)
        blocks[er] = 0x5C
        O.poly_decode(w, k, m, er, blocks)
        assert np.array_equal(blocks, ref), (stripe, er)


def test_decode_rejects_bad_erasures():
    blocks = np.zeros((14, 8), dtype=np.uint8)
    with pytest.raises(ValueError):
        O.poly_decode(8, 10, 4, [0, 1, 2, 3, 4], blocks)  # e > m
    with pytest.raises(ValueError):
        O.poly_decode(8, 10, 4, [1, 1], blocks)  # duplicate
    with pytest.raises(ValueError):
        O.poly_decode(8, 10, 4, [14], blocks)  # out of range


# ---------------------------------------------------- GF(2^4) brute force
def _gf16_codes():
    for n in range(2, 16):
        for m in range(1, n):
            yield n - m, m


@pytest.mark.parametrize("realization", ["poly", "vandermonde"])
def test_gf16_all_codes_all_erasure_patterns(realization):
    """Every (k, m) with n <= 15 in GF(2^4): every erasure pattern of every
    size e <= m is recovered exactly (capped per code for run time)."""
    w = 4
    rng = np.random.default_rng(2024)
    total = 0
    for k, m in _gf16_codes():
        n = k + m
        B = 6
        blocks = np.zeros((n, B), dtype=np.uint8)
        blocks[:k] = rng.integers(0, 16, (k, B), dtype=np.uint8)
        O.encode(realization, w, k, m, blocks)
        ref = blocks.copy()
        pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
        if len(pats) > 400:
            idx = rng.choice(len(pats), 400, replace=False)
            pats = [pats[i] for i in idx]
        for p in pats:
            x = ref.copy()
            x[list(p)] = 0
            O.decode(realization, w, k, m, list(p), x)
            assert np.array_equal(x, ref), (k, m, p)
            total += 1
    assert total > 10_000
