"""Pins of the oracle's generator-matrix forms of the polynomial code (§6):
the parity matrix P (column i = x^(m+i) mod g(x)) in the symbol layout and
its bit-matrix (packet-layout) projection."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests import gfref
from tests.test_oracle_poly import read_golden


def test_worked_example_through_the_generator_matrix():
    """P times the §3.2 example data gives the example's parity."""
    g = read_golden()
    Pm = O.polymat_matrix(8, 4, 3)
    d = g["data"]
    p = []
    for j in range(3):
        s = 0
        for i in range(4):
            s ^= gfref.mul(int(Pm[j, i]), d[i], 8)
        p.append(s)
    assert p == g["parity"]


@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (16, 12, 4), (8, 5, 7)])
def test_generator_matrix_codewords_have_the_roots(w, k, m):
    Pm = O.polymat_matrix(w, k, m)
    rng = np.random.default_rng(w * 100 + k)
    d = [int(x) for x in rng.integers(0, 1 << w, k)]
    p = []
    for j in range(m):
        s = 0
        for i in range(k):
            s ^= gfref.mul(int(Pm[j, i]), d[i], w)
        p.append(s)
    coeffs = p + d  # parity at x^0..x^(m-1), data at x^m..
    a = 1
    for _ in range(m):
        assert gfref.poly_eval(coeffs, a, w) == 0
        a = gfref.mul(a, 2, w)


@pytest.mark.parametrize("w,k,m,P", [(8, 10, 4, 16), (8, 6, 3, 8), (16, 12, 4, 8)])
def test_bitmatrix_form_read_as_symbols_is_the_polynomial_code(w, k, m, P):
    B = 2 * w * P
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(51, 0, k, B)
    O.polybm_encode(w, k, m, blocks, P)
    dsym = np.stack([gfref.packets_to_symbols(blocks[j], w, P) for j in range(k)])
    psym = np.stack([gfref.packets_to_symbols(blocks[k + i], w, P) for i in range(m)])
    for t in range(0, dsym.shape[1], 7):
        assert O.poly_encode_column(w, k, m, dsym[:, t]).tolist() == psym[:, t].tolist()


@pytest.mark.parametrize("w,k,m,P", [(8, 6, 3, 8), (8, 10, 4, 16), (4, 5, 3, 4)])
def test_bitmatrix_form_round_trip(w, k, m, P):
    n = k + m
    B = 2 * w * P
    blocks = np.zeros((n, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(52, 0, k, B)
    O.polybm_encode(w, k, m, blocks, P)
    ref = blocks.copy()
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    if len(pats) > 250:
        rng = np.random.default_rng(4)
        pats = [pats[i] for i in rng.choice(len(pats), 250, replace=False)]
    for pat in pats:
        x = ref.copy()
        x[list(pat)] = 0x81
        O.polybm_decode(w, k, m, list(pat), x, P)
        assert np.array_equal(x, ref), pat
