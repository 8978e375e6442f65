"""Pins of the oracle's matrix realizations (§2).

Vandermonde (§2.2): the systematic generator must produce, for data d, the
values at points k..n-1 of the polynomial of degree < k through
(0, d_0) .. (k-1, d_{k-1}); checked with Lagrange interpolation.  Every k x k
submatrix of the generator must be invertible (§2.1).
Cauchy (§2.3): entries 1/(x_i + y_j); the bit-matrix M(e) is the matrix of
x -> e x over GF(2); parity read back through the packet layout equals the
GF(2^w) product C d.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests import gfref


# ------------------------------------------------------------ Vandermonde
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (16, 12, 4), (4, 5, 3)])
def test_vandermonde_is_systematic(w, k, m):
    G = O.vand_matrix(w, k, m)
    assert np.array_equal(G[:k], np.eye(k, dtype=np.uint32))


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (16, 12, 4)])
def test_vandermonde_parity_is_interpolation(w, k, m):
    B = 4 if w == 16 else 2
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(77, 0, k, B)
    O.vand_encode(w, k, m, blocks)
    syms = np.stack([gfref.symbols(blocks[b], w) for b in range(k + m)])
    xs = list(range(k))
    for t in range(syms.shape[1]):
        ys = [int(v) for v in syms[:k, t]]
        for j in range(m):
            assert int(syms[k + j, t]) == gfref.lagrange_eval(xs, ys, k + j, w), (t, j)


def test_vandermonde_rs_10_4_every_k_subset_invertible():
    w, k, m = 8, 10, 4
    G = O.vand_matrix(w, k, m).tolist()
    for rows in itertools.combinations(range(k + m), k):
        assert gfref.rank([G[r] for r in rows], w) == k, rows


@pytest.mark.parametrize("w,k,m", [(8, 6, 3), (8, 10, 4), (16, 12, 4)])
def test_vandermonde_round_trip(w, k, m):
    n = k + m
    B = 16
    blocks = np.zeros((n, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(31, 0, k, B)
    O.vand_encode(w, k, m, blocks)
    ref = blocks.copy()
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    if len(pats) > 300:
        rng = np.random.default_rng(3)
        pats = [pats[i] for i in rng.choice(len(pats), 300, replace=False)]
    for p in pats:
        x = ref.copy()
        x[list(p)] = 0x77
        O.vand_decode(w, k, m, list(p), x)
        assert np.array_equal(x, ref), p


# ----------------------------------------------------------------- Cauchy
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (16, 12, 4), (8, 20, 4)])
def test_cauchy_entries_are_reciprocals(w, k, m):
    C = O.cauchy_matrix(w, k, m)
    for i in range(m):
        for j in range(k):
            assert gfref.mul(int(C[i, j]), i ^ (m + j), w) == 1


@pytest.mark.parametrize("w", [4, 8])
def test_bitmatrix_is_multiplication_map_all_elements(w):
    q = 1 << w
    xs = np.arange(q, dtype=np.uint32)
    xbits = ((xs[:, None] >> np.arange(w, dtype=np.uint32)) & 1).astype(np.uint8)  # (q, w)
    for e in range(q):
        M = O.bitmatrix(w, e).astype(np.uint8)
        ybits = (xbits @ M.T) & 1  # row x: M * bits(x)
        y = (ybits.astype(np.uint32) << np.arange(w, dtype=np.uint32)).sum(axis=1)
        assert np.array_equal(y, gfref.mul_np(e, xs, w)), e


def test_bitmatrix_w16_sampled():
    rng = np.random.default_rng(5)
    xs = rng.integers(0, 1 << 16, 512, dtype=np.uint32)
    xbits = ((xs[:, None] >> np.arange(16, dtype=np.uint32)) & 1).astype(np.int64)
    for e in [1, 2, 0x100B, 0xFFFF, 12345, 40000]:
        M = O.bitmatrix(16, e).astype(np.int64)
        y = (((xbits @ M.T) & 1) << np.arange(16)).sum(axis=1).astype(np.uint32)
        assert np.array_equal(y, gfref.mul_np(e, xs, 16))


@pytest.mark.parametrize("w,k,m,P", [(8, 10, 4, 16), (8, 6, 3, 8), (16, 12, 4, 8)])
def test_cauchy_packets_read_as_symbols_equal_matrix_product(w, k, m, P):
    B = 2 * w * P
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(41, 0, k, B)
    O.cauchy_encode(w, k, m, blocks, P)
    C = O.cauchy_matrix(w, k, m)
    dsym = np.stack([gfref.packets_to_symbols(blocks[j], w, P) for j in range(k)])
    for i in range(m):
        psym = gfref.packets_to_symbols(blocks[k + i], w, P)
        want = np.zeros_like(psym)
        for j in range(k):
            want ^= gfref.mul_np(int(C[i, j]), dsym[j], w)
        assert np.array_equal(psym, want), i


@pytest.mark.parametrize("w,k,m,P", [(8, 6, 3, 8), (8, 10, 4, 16), (16, 12, 4, 4), (4, 5, 3, 4)])
def test_cauchy_round_trip(w, k, m, P):
    n = k + m
    B = 2 * w * P
    blocks = np.zeros((n, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(43, 0, k, B)
    O.cauchy_encode(w, k, m, blocks, P)
    ref = blocks.copy()
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    if len(pats) > 250:
        rng = np.random.default_rng(9)
        pats = [pats[i] for i in rng.choice(len(pats), 250, replace=False)]
    for p in pats:
        x = ref.copy()
        x[list(p)] = 0x3C
        O.cauchy_decode(w, k, m, list(p), x, P)
        assert np.array_equal(x, ref), p


def test_generators_agree_on_the_mds_property_small_field():
    """GF(2^4), every (k, m) with n <= 15: every k-subset of rows of the
    systematic Vandermonde and Cauchy generators has full rank."""
    w = 4
    rng = np.random.default_rng(0)
    for n in range(3, 16):
        for m in range(1, min(n, 5)):
            k = n - m
            Gv = O.vand_matrix(w, k, m).tolist()
            C = O.cauchy_matrix(w, k, m).tolist()
            Gc = [[int(r == c) for c in range(k)] for r in range(k)] + C
            subsets = list(itertools.combinations(range(n), k))
            if len(subsets) > 60:
                subsets = [subsets[i] for i in rng.choice(len(subsets), 60, replace=False)]
            for rows in subsets:
                assert gfref.rank([Gv[r] for r in rows], w) == k
                assert gfref.rank([Gc[r] for r in rows], w) == k
