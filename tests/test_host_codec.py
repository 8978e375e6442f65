"""CPU checks of the library's bit-sliced codecs and decode planner.

tests/hostemu builds the library's own codec templates and plan.cpp for the
host (the GPU kernels run the same templates), so the arithmetic and the
plans are compared with the oracle here, without a GPU.
"""
import ctypes
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests.hostemu.build import build

U8P = ctypes.POINTER(ctypes.c_uint8)


@pytest.fixture(scope="module")
def emu():
    L = build()
    L.emu_poly_encode.argtypes = [ctypes.c_int] * 3 + [U8P, ctypes.c_size_t]
    L.emu_poly_decode.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                       ctypes.c_int, U8P, ctypes.c_size_t]
    L.emu_genpoly.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
    L.emu_transpose.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
    return L


def _enc(L, w, k, m, blocks):
    assert L.emu_poly_encode(w, k, m, blocks.ctypes.data_as(U8P), blocks.shape[1]) == 0


def _dec(L, w, k, m, er, blocks, read_all):
    arr = (ctypes.c_int * max(1, len(er)))(*er)
    assert L.emu_poly_decode(w, k, m, arr, len(er), int(read_all), blocks.ctypes.data_as(U8P),
                             blocks.shape[1]) == 0


@pytest.mark.parametrize("w", [8, 16])
@pytest.mark.parametrize("m", range(1, 9))
def test_compile_time_generator_matches_oracle(emu, w, m):
    g = (ctypes.c_uint32 * 9)()
    emu.emu_genpoly(w, m, g)
    assert list(g)[:m + 1] == O.genpoly(w, m).tolist()


@pytest.mark.parametrize("w", [8, 16])
def test_transpose_is_an_involution_and_slices_bits(emu, w):
    rng = np.random.default_rng(w)
    x = rng.integers(0, 2**32, w, dtype=np.uint64).astype(np.uint32)
    y = x.copy()
    emu.emu_transpose(w, y.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    # plane b holds bit b of every symbol: count of set bits per plane equals
    # the number of symbols with bit b set
    per_word = 32 // w
    syms = [(int(x[v]) >> (w * i)) & ((1 << w) - 1) for v in range(w) for i in range(per_word)]
    for b in range(w):
        assert bin(int(y[b])).count("1") == sum((s >> b) & 1 for s in syms)
    z = y.copy()
    emu.emu_transpose(w, z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert np.array_equal(z, x)


ENC_CASES = [(8, 10, 4, 65536), (8, 10, 4, 1000), (8, 6, 3, 4096 + 16), (8, 20, 4, 3000),
             (8, 3, 8, 2048), (8, 5, 5, 777), (8, 1, 1, 33), (16, 12, 4, 8192), (16, 12, 4, 2050),
             (16, 4, 7, 600), (8, 10, 4, 0 + 16), (8, 2, 2, 1)]


@pytest.mark.parametrize("w,k,m,B", ENC_CASES)
def test_encode_matches_oracle(emu, w, k, m, B):
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(inputs.stream_seed(1), 0, k, B)
    ref = blocks.copy()
    O.poly_encode(w, k, m, ref)
    got = blocks.copy()
    got[k:] = 0x5A
    _enc(emu, w, k, m, got)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("w,k,m", [(8, 6, 3), (8, 4, 4), (16, 5, 3)])
def test_decode_every_pattern_small_codes(emu, w, k, m, read_all):
    n, B = k + m, 2048 + 48
    blocks = np.zeros((n, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(17, 0, k, B)
    O.poly_encode(w, k, m, blocks)
    for e in range(1, m + 1):
        for er in itertools.combinations(range(n), e):
            got = blocks.copy()
            got[list(er)] = 0xEE
            _dec(emu, w, k, m, list(er), got, read_all)
            assert np.array_equal(got, blocks), er


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (16, 12, 4), (8, 20, 4), (8, 10, 6)])
def test_decode_seeded_patterns_match_oracle(emu, w, k, m, read_all):
    n, B = k + m, 4096 + 32
    seed = inputs.stream_seed(2)
    for stripe in range(6):
        blocks = np.zeros((n, B), dtype=np.uint8)
        blocks[:k] = inputs.stripe_blocks(seed, stripe, k, B)
        O.poly_encode(w, k, m, blocks)
        e = 1 + stripe % m
        er = inputs.erasure_pattern(seed, stripe, n, e)
        ref = blocks.copy()
        ref[er] = 0
        O.poly_decode(w, k, m, er, ref)
        got = blocks.copy()
        got[er] = 0x11
        _dec(emu, w, k, m, er, got, read_all)
        assert np.array_equal(got, ref), er


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("k,m,B", [(10, 4, 4096 + 48), (6, 3, 3000), (12, 4, 2048 + 7), (5, 2, 2048),
                                   (20, 4, 9000), (3, 1, 100), (10, 5, 3000), (10, 6, 2048 + 9)])
def test_two_group_decode_matches_oracle(emu, k, m, B, read_all):
    """The decode with two 32-column groups per thread (GF(2^8), M <= 6;
    two selector chunks for M = 5, 6)."""
    emu.emu_poly_decode2.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                          ctypes.c_int, U8P, ctypes.c_size_t]
    w, n = 8, k + m
    base = np.zeros((n, B), dtype=np.uint8)
    base[:k] = inputs.stripe_blocks(23, 0, k, B)
    O.poly_encode(w, k, m, base)
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    rng = np.random.default_rng(k * 100 + m)
    if len(pats) > 40:
        pats = [pats[i] for i in rng.choice(len(pats), 40, replace=False)]
    for er in pats:
        got = base.copy()
        got[list(er)] = 0x5A
        arr = (ctypes.c_int * len(er))(*er)
        rc = emu.emu_poly_decode2(w, k, m, arr, len(er), int(read_all), got.ctypes.data_as(U8P), B)
        if rc == -2:  # M > 6
            continue
        assert rc == 0
        assert np.array_equal(got, base), er


@pytest.mark.parametrize("real,k,m,B", [("vandermonde", 10, 4, 4096 + 16), ("vandermonde", 6, 3, 3000),
                                        ("poly_matrix", 10, 4, 5000), ("poly_matrix", 10, 4, 100)])
def test_two_group_encode_matches_oracle(emu, real, k, m, B):
    """The compile-time-P encodes with two 32-column groups per thread."""
    emu.emu_encode2.argtypes = [ctypes.c_int] * 3 + [U8P, ctypes.c_size_t]
    kind = {"vandermonde": 1, "poly_matrix": 3}[real]
    w = 8
    base = np.zeros((k + m, B), dtype=np.uint8)
    base[:k] = inputs.stripe_blocks(29, 0, k, B)
    ref = base.copy()
    O.encode(real, w, k, m, ref)
    got = base.copy()
    got[k:] = 0x3C
    assert emu.emu_encode2(kind, k, m, got.ctypes.data_as(U8P), B) == 0
    assert np.array_equal(got, ref)
