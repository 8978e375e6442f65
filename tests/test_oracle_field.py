"""Pins of the oracle's GF(2^w) tables against the field's definition.

The oracle multiplies through exp/log tables; these tests compare it with the
table-free shift-and-add product of tests/gfref.py and with field axioms.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import gfref


@pytest.mark.parametrize("w", [4, 8])
def test_mul_all_pairs_match_shift_and_add(w):
    q = 1 << w
    a, b = np.meshgrid(np.arange(q, dtype=np.uint32), np.arange(q, dtype=np.uint32), indexing="ij")
    got = O.gf_mul(w, a.ravel(), b.ravel())
    want = gfref.mul_np(a.ravel(), b.ravel(), w)
    assert np.array_equal(got, want)


def test_w4_associative_distributive_exhaustive():
    w, q = 4, 16
    x = np.arange(q, dtype=np.uint32)
    a, b, c = [t.ravel() for t in np.meshgrid(x, x, x, indexing="ij")]
    ab_c = O.gf_mul(w, O.gf_mul(w, a, b), c)
    a_bc = O.gf_mul(w, a, O.gf_mul(w, b, c))
    assert np.array_equal(ab_c, a_bc)
    left = O.gf_mul(w, a, b ^ c)
    right = O.gf_mul(w, a, b) ^ O.gf_mul(w, a, c)
    assert np.array_equal(left, right)
    assert np.array_equal(O.gf_mul(w, a, b), O.gf_mul(w, b, a))


@pytest.mark.parametrize("w", [4, 8, 16])
def test_inverse_of_every_nonzero_element(w):
    a = np.arange(1, 1 << w, dtype=np.uint32)
    ia = O.gf_inv(w, a)
    assert np.all(O.gf_mul(w, a, ia) == 1)
    # spot check against Fermat inversion (a^(2^w-2)) for a spread of elements
    for v in list(range(1, min(1 << w, 64))) + [(1 << w) - 1, (1 << w) // 2 + 3]:
        assert int(ia[v - 1]) == gfref.inv(v, w)


@pytest.mark.parametrize("w", [4, 8, 16])
def test_alpha_two_is_primitive(w):
    """exp table = successive powers of 2: all 2^w - 1 nonzero values, once each."""
    ex = O.gf_exp_table(w)
    assert ex[0] == 1
    assert len(np.unique(ex)) == (1 << w) - 1
    assert ex.min() == 1 and ex.max() == (1 << w) - 1
    # consecutive entries differ by a factor alpha = 2 (shift-and-add product)
    assert np.array_equal(gfref.mul_np(ex[:-1], 2, w), ex[1:])
    assert gfref.mul(int(ex[-1]), 2, w) == 1


def test_w16_random_products_match_shift_and_add():
    rng = np.random.default_rng(1234)
    a = rng.integers(0, 1 << 16, 200_000, dtype=np.uint32)
    b = rng.integers(0, 1 << 16, 200_000, dtype=np.uint32)
    assert np.array_equal(O.gf_mul(16, a, b), gfref.mul_np(a, b, 16))


def test_alpha8_is_29_in_gf256():
    """§3.3's example matrix writes alpha^8 as 29, which fixes the
    primitive polynomial 0x11D among those with alpha = 2 primitive."""
    ex = O.gf_exp_table(8)
    assert int(ex[8]) == 29
    assert int(ex[10]) == 116 and int(ex[5]) == 32 and int(ex[6]) == 64


def test_invert_matrix_roundtrip():
    rng = np.random.default_rng(7)
    for w in (8, 16):
        for n in (1, 2, 4, 7):
            while True:
                A = rng.integers(0, 1 << w, (n, n)).astype(np.uint32)
                if gfref.rank(A.tolist(), w) == n:
                    break
            Ai = O.gf_invert_matrix(w, A)
            # product with independent arithmetic is the identity
            for r in range(n):
                for c in range(n):
                    s = 0
                    for t in range(n):
                        s ^= gfref.mul(int(A[r, t]), int(Ai[t, c]), w)
                    assert s == (1 if r == c else 0)
