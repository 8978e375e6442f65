"""Pins of the oracle's "good" Cauchy matrices (§2.3: Cauchy matrices differ
in efficiency, the XOR count of the bit-matrix code being the number of ones
of its projection; the paper benchmarks such matrices as GoodCRS, §5.1).

Reading (the paper gives no construction): the original Cauchy matrix with
every column divided by its row-0 entry, then every other row divided by
the divisor (1 or one of the row's entries) that leaves the fewest ones.
The pins check, with arithmetic independent of the oracle (tests/gfref.py):
the code stays MDS (every k-subset of the generator's rows has full rank),
each row is the original row scaled by nonzero constants of the stated
form, no candidate divisor beats the chosen one, the matrix has no more
ones than the original, and the packet-layout code computes C d."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests import gfref


def ones(e: int, w: int) -> int:
    """Ones of the §2.3 projection of e: column c is e * alpha^c."""
    return sum(bin(gfref.mul(e, gfref.power(2, c, w), w)).count("1") for c in range(w))


@pytest.mark.parametrize("w", [4, 8, 16])
def test_ones_count_matches_independent_projection(w):
    for e in [1, 2, 3, 0x1D, (1 << w) - 1, 5, 7 % (1 << w)]:
        e %= 1 << w
        if e:
            assert O.bitmatrix_ones(w, e) == ones(e, w)
    assert O.bitmatrix_ones(w, 1) == w  # the identity


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (16, 12, 4), (8, 20, 4), (4, 5, 3)])
def test_good_cauchy_is_a_scaling_of_the_original(w, k, m):
    C = O.cauchy_matrix(w, k, m).tolist()
    G = O.goodcauchy_matrix(w, k, m).tolist()
    assert G[0] == [1] * k  # row 0 normalised to ones
    for i in range(1, m):
        # G[i][j] = C[i][j] / (C[0][j] * r_i): the same r_i for every column
        r = {gfref.mul(gfref.mul(C[i][j], gfref.inv(C[0][j], w), w), gfref.inv(G[i][j], w), w) for j in range(k)}
        assert len(r) == 1 and 0 not in r, (i, r)


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (4, 5, 3), (16, 12, 4)])
def test_good_cauchy_rows_take_the_best_divisor(w, k, m):
    C = O.cauchy_matrix(w, k, m).tolist()
    G = O.goodcauchy_matrix(w, k, m).tolist()
    for i in range(1, m):
        # the column-normalised row, then every candidate divisor
        base = [gfref.mul(C[i][j], gfref.inv(C[0][j], w), w) for j in range(k)]
        cands = [1] + base
        cost = [sum(ones(gfref.mul(x, gfref.inv(v, w), w), w) for x in base) for v in cands]
        assert sum(ones(x, w) for x in G[i]) == min(cost), i
    total_good = sum(ones(x, w) for row in G for x in row)
    total_orig = sum(ones(x, w) for row in C for x in row)
    assert total_good <= total_orig


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3)])
def test_good_cauchy_every_k_subset_invertible(w, k, m):
    G = O.goodcauchy_matrix(w, k, m).tolist()
    gen = [[int(r == c) for c in range(k)] for r in range(k)] + G
    for rows in itertools.combinations(range(k + m), k):
        assert gfref.rank([gen[r] for r in rows], w) == k, rows


def test_good_cauchy_mds_small_field_every_code():
    """GF(2^4), every (k, m) with n <= 15 and m <= 4: every k-subset of the
    systematic generator's rows has full rank (sampled above 60 subsets)."""
    w = 4
    rng = np.random.default_rng(1)
    for n in range(3, 16):
        for m in range(1, min(n, 5)):
            k = n - m
            gen = [[int(r == c) for c in range(k)] for r in range(k)] + O.goodcauchy_matrix(w, k, m).tolist()
            subsets = list(itertools.combinations(range(n), k))
            if len(subsets) > 60:
                subsets = [subsets[i] for i in rng.choice(len(subsets), 60, replace=False)]
            for rows in subsets:
                assert gfref.rank([gen[r] for r in rows], w) == k, (k, m, rows)


@pytest.mark.parametrize("w,k,m,P", [(8, 10, 4, 16), (8, 6, 3, 8), (16, 12, 4, 8)])
def test_good_cauchy_packets_read_as_symbols_equal_matrix_product(w, k, m, P):
    B = 2 * w * P
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(47, 0, k, B)
    O.goodcauchy_encode(w, k, m, blocks, P)
    G = O.goodcauchy_matrix(w, k, m)
    dsym = np.stack([gfref.packets_to_symbols(blocks[j], w, P) for j in range(k)])
    for i in range(m):
        psym = gfref.packets_to_symbols(blocks[k + i], w, P)
        want = np.zeros_like(psym)
        for j in range(k):
            want ^= gfref.mul_np(int(G[i, j]), dsym[j], w)
        assert np.array_equal(psym, want), i


@pytest.mark.parametrize("w,k,m,P", [(8, 6, 3, 8), (8, 10, 4, 16), (16, 12, 4, 4), (4, 5, 3, 4)])
def test_good_cauchy_round_trip(w, k, m, P):
    n = k + m
    B = 2 * w * P
    blocks = np.zeros((n, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(53, 0, k, B)
    O.goodcauchy_encode(w, k, m, blocks, P)
    ref = blocks.copy()
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    if len(pats) > 250:
        rng = np.random.default_rng(11)
        pats = [pats[i] for i in rng.choice(len(pats), 250, replace=False)]
    for p in pats:
        x = ref.copy()
        x[list(p)] = 0x5A
        O.goodcauchy_decode(w, k, m, list(p), x, P)
        assert np.array_equal(x, ref), p
