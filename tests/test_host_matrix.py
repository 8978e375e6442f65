"""CPU checks of the library's matrix-realization codecs (Vandermonde in
the symbol layout, Cauchy in the packet layout), compile-time and runtime P,
against the oracle."""
import ctypes
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests.hostemu.build import build

U8P = ctypes.POINTER(ctypes.c_uint8)
KIND = {"vandermonde": 1, "cauchy": 2, "poly_matrix": 3, "poly_bitmatrix": 4, "good_cauchy": 5}
FIXED = {(8, 6, 3), (8, 10, 4), (8, 12, 4), (8, 20, 4), (16, 12, 4)}
FIXED_POLY = {(8, 10, 4), (8, 6, 3), (16, 12, 4)}  # harness instantiations of kinds 3 and 4


@pytest.fixture(scope="module")
def emu():
    L = build()
    L.emu_mat.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, U8P,
                                               ctypes.c_size_t, ctypes.c_size_t]
    L.emu_parity_matrix.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_uint32)]
    L.emu_fixed_parity_matrix.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_uint32)]
    return L


def run(L, real, w, k, m, fixed, er, blocks, pkt, read_all=False):
    arr = (ctypes.c_int * max(1, len(er)))(*er)
    rc = L.emu_mat(w, k, m, KIND[real], int(fixed), arr, len(er), int(read_all), blocks.ctypes.data_as(U8P),
                   blocks.shape[1], pkt)
    assert rc == 0, rc


def oracle_parity(real, w, k, m):
    if real == "vandermonde":
        return O.vand_matrix(w, k, m)[k:]
    if real == "cauchy":
        return O.cauchy_matrix(w, k, m)
    if real == "good_cauchy":
        return O.goodcauchy_matrix(w, k, m)
    return O.polymat_matrix(w, k, m)


@pytest.mark.parametrize("real", ["vandermonde", "cauchy", "poly_matrix", "good_cauchy"])
@pytest.mark.parametrize("w,k,m", [(8, 10, 4), (8, 6, 3), (16, 12, 4), (8, 5, 7), (8, 20, 4), (16, 3, 2)])
def test_host_parity_matrix_matches_oracle(emu, real, w, k, m):
    out = (ctypes.c_uint32 * (k * m))()
    assert emu.emu_parity_matrix(w, k, m, KIND[real], out) == 0
    got = np.array(list(out), dtype=np.uint32).reshape(m, k)
    assert np.array_equal(got, oracle_parity(real, w, k, m))


@pytest.mark.parametrize("real", ["vandermonde", "cauchy", "poly_matrix", "good_cauchy"])
@pytest.mark.parametrize("w,k,m", [(8, 6, 3), (8, 10, 4), (8, 12, 4), (8, 20, 4), (16, 12, 4)])
def test_compile_time_parity_matrix_matches_oracle(emu, real, w, k, m):
    """The compile-time (constexpr) generators the fixed-code kernels are
    built from equal the oracle's matrices for every compiled code."""
    out = (ctypes.c_uint32 * (k * m))()
    assert emu.emu_fixed_parity_matrix(w, k, m, KIND[real], out) == 0
    got = np.array(list(out), dtype=np.uint32).reshape(m, k)
    assert np.array_equal(got, oracle_parity(real, w, k, m))


def make_stripe(w, k, m, B, seed=3, stripe=0):
    blocks = np.zeros((k + m, B), dtype=np.uint8)
    blocks[:k] = inputs.stripe_blocks(seed, stripe, k, B)
    return blocks


CASES = [("vandermonde", 8, 10, 4, 4096 + 48, 0), ("vandermonde", 8, 6, 3, 3000, 0),
         ("vandermonde", 16, 12, 4, 8192 + 2, 0), ("vandermonde", 8, 5, 7, 2048, 0),
         ("vandermonde", 8, 20, 4, 1100, 0),
         ("cauchy", 8, 10, 4, 8 * 256 * 2, 256), ("cauchy", 8, 6, 3, 8 * 128 * 3, 128),
         ("cauchy", 16, 12, 4, 16 * 128 * 2, 128), ("cauchy", 8, 5, 7, 8 * 384, 384),
         ("cauchy", 8, 20, 4, 8 * 128, 128),
         ("poly_matrix", 8, 10, 4, 4096 + 48, 0), ("poly_matrix", 8, 6, 3, 3000, 0),
         ("poly_matrix", 16, 12, 4, 8192 + 2, 0), ("poly_matrix", 8, 5, 7, 2048, 0),
         ("poly_bitmatrix", 8, 10, 4, 8 * 256 * 2, 256), ("poly_bitmatrix", 8, 6, 3, 8 * 128 * 3, 128),
         ("poly_bitmatrix", 16, 12, 4, 16 * 128 * 2, 128), ("poly_bitmatrix", 8, 5, 7, 8 * 384, 384),
         ("good_cauchy", 8, 10, 4, 8 * 256 * 2, 256), ("good_cauchy", 8, 6, 3, 8 * 128 * 3, 128),
         ("good_cauchy", 16, 12, 4, 16 * 128 * 2, 128), ("good_cauchy", 8, 5, 7, 8 * 384, 384),
         ("good_cauchy", 8, 20, 4, 8 * 128, 128)]


def fixed_ok(real, w, k, m):
    return (w, k, m) in (FIXED_POLY if real.startswith("poly") else FIXED)


@pytest.mark.parametrize("real,w,k,m,B,pkt", CASES)
def test_encode_matches_oracle(emu, real, w, k, m, B, pkt):
    base = make_stripe(w, k, m, B)
    ref = base.copy()
    O.encode(real, w, k, m, ref, packet_bytes=pkt or 2048)
    for fixed in (False, True):
        if fixed and not fixed_ok(real, w, k, m):
            continue
        got = base.copy()
        got[k:] = 0x44
        run(emu, real, w, k, m, fixed, [], got, pkt)
        assert np.array_equal(got, ref), fixed


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("real,w,k,m,B,pkt", CASES)
def test_decode_seeded_patterns(emu, real, w, k, m, B, pkt, read_all):
    base = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, base, packet_bytes=pkt or 2048)
    n = k + m
    for stripe in range(2 * m):
        e = 1 + stripe % m
        er = inputs.erasure_pattern(11, stripe, n, e)
        for fixed in (False, True):
            if fixed and not fixed_ok(real, w, k, m):
                continue
            got = base.copy()
            got[er] = 0x99
            run(emu, real, w, k, m, fixed, er, got, pkt, read_all)
            assert np.array_equal(got, base), (er, fixed)


@pytest.mark.parametrize("real", ["vandermonde", "cauchy", "poly_matrix", "poly_bitmatrix", "good_cauchy"])
def test_decode_every_pattern_rs_6_3(emu, real):
    w, k, m = 8, 6, 3
    pkt = 128
    B = 8 * pkt
    base = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, base, packet_bytes=pkt)
    n = k + m
    for e in range(1, m + 1):
        for er in itertools.combinations(range(n), e):
            for fixed in (False, True):
                got = base.copy()
                got[list(er)] = 0
                run(emu, real, w, k, m, fixed, list(er), got, pkt, read_all=(e % 2 == 0))
                assert np.array_equal(got, base), (er, fixed)


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("real,k,m,B", [("vandermonde", 10, 4, 4096 + 48), ("vandermonde", 6, 3, 3000),
                                        ("vandermonde", 20, 4, 2048 + 5), ("poly_matrix", 10, 4, 3000),
                                        ("poly_matrix", 6, 3, 100)])
def test_two_group_matrix_decode_matches_oracle(emu, real, k, m, B, read_all):
    """The compile-time-P decode with two 32-column groups per thread."""
    emu.emu_mat_decode2.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                                         U8P, ctypes.c_size_t]
    w, n = 8, k + m
    base = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, base)
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    rng = np.random.default_rng(k * 10 + m)
    if len(pats) > 40:
        pats = [pats[i] for i in rng.choice(len(pats), 40, replace=False)]
    for er in pats:
        got = base.copy()
        got[list(er)] = 0x77
        arr = (ctypes.c_int * len(er))(*er)
        rc = emu.emu_mat_decode2(w, k, m, KIND[real], arr, len(er), int(read_all), got.ctypes.data_as(U8P), B)
        assert rc == 0, rc
        assert np.array_equal(got, base), er


@pytest.mark.parametrize("read_all", [False, True])
@pytest.mark.parametrize("real,k,m,pkt,sp", [("cauchy", 10, 4, 256, 3), ("cauchy", 6, 3, 2048, 1),
                                             ("poly_bitmatrix", 10, 4, 512, 2), ("good_cauchy", 10, 4, 256, 3),
                                             ("good_cauchy", 6, 3, 2048, 1)])
def test_two_group_packet_decode_matches_oracle(emu, real, k, m, pkt, sp, read_all):
    """The packet-layout compile-time-P decode with two adjacent words per
    thread (one 64-bit load per packet row)."""
    emu.emu_mat_decode2_packet.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                                ctypes.c_int, U8P, ctypes.c_size_t, ctypes.c_size_t]
    w, n = 8, k + m
    B = sp * w * pkt
    base = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, base, packet_bytes=pkt)
    pats = [p for e in range(1, m + 1) for p in itertools.combinations(range(n), e)]
    rng = np.random.default_rng(k * 100 + m + pkt)
    if len(pats) > 30:
        pats = [pats[i] for i in rng.choice(len(pats), 30, replace=False)]
    for er in pats:
        got = base.copy()
        got[list(er)] = 0x5A
        arr = (ctypes.c_int * len(er))(*er)
        rc = emu.emu_mat_decode2_packet(w, k, m, KIND[real], arr, len(er), int(read_all), got.ctypes.data_as(U8P),
                                        B, pkt)
        assert rc == 0, rc
        assert np.array_equal(got, base), er


@pytest.mark.parametrize("real,pkt,sp", [("cauchy", 256, 2), ("good_cauchy", 2048, 1), ("good_cauchy", 128, 3)])
def test_gf16_two_group_packet_encode_matches_oracle(emu, real, pkt, sp):
    """The GF(2^16) packet-layout encode with two adjacent words per thread
    (the kernel that covers a whole super-packet per tile)."""
    emu.emu_mat_encode2_packet.argtypes = [ctypes.c_int] * 4 + [U8P, ctypes.c_size_t, ctypes.c_size_t]
    w, k, m = 16, 12, 4
    B = sp * w * pkt
    ref = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, ref, packet_bytes=pkt)
    got = ref.copy()
    got[k:] = 0xA5
    rc = emu.emu_mat_encode2_packet(w, k, m, KIND[real], got.ctypes.data_as(U8P), B, pkt)
    assert rc == 0, rc
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("real,pkt,sp", [("cauchy", 256, 1), ("good_cauchy", 128, 2)])
def test_gf16_two_group_packet_decode_matches_oracle(emu, real, pkt, sp):
    """The GF(2^16) packet-layout decode with two adjacent words per thread
    (no pair sums): every erasure count, min-read and read-all."""
    emu.emu_mat_decode2_packet.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                                ctypes.c_int, U8P, ctypes.c_size_t, ctypes.c_size_t]
    w, k, m = 16, 12, 4
    n = k + m
    B = sp * w * pkt
    base = make_stripe(w, k, m, B)
    O.encode(real, w, k, m, base, packet_bytes=pkt)
    rng = np.random.default_rng(pkt + sp)
    for e in range(1, m + 1):
        for read_all in (False, True):
            er = sorted(int(x) for x in rng.choice(n, e, replace=False))
            got = base.copy()
            got[er] = 0x3C
            arr = (ctypes.c_int * e)(*er)
            rc = emu.emu_mat_decode2_packet(w, k, m, KIND[real], arr, e, int(read_all), got.ctypes.data_as(U8P), B,
                                            pkt)
            assert rc == 0, rc
            assert np.array_equal(got, base), (er, read_all)
