"""GPU parity: Vandermonde (symbol layout) and Cauchy bit-matrix (packet
layout; original and "good" Cauchy matrices) realizations through the C ABI
vs the CPU oracle, bit-exact.
Registered codes run the compile-time-generator kernels, other codes the
runtime-generator kernels; both are covered."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests.gpu_util import device_blocks, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs as rsmod
    build.build()
    return rsmod


def stripe(w, k, m, B, seed=7, s=0):
    host = np.zeros((k + m, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(inputs.stream_seed(seed), s, k, B)
    return host


# (realization, w, k, m, B, packet)
CASES = [
    ("vandermonde", 8, 10, 4, 1 << 20, None), ("vandermonde", 8, 10, 4, 65536 + 37, None),
    ("vandermonde", 8, 6, 3, 300000, None), ("vandermonde", 16, 12, 4, 100002, None),
    ("vandermonde", 8, 20, 4, 8192, None), ("vandermonde", 8, 7, 5, 50000, None),
    ("vandermonde", 16, 5, 3, 4096 + 2, None), ("vandermonde", 8, 10, 4, (1 << 18) + 37, None),
    ("vandermonde", 8, 12, 4, (1 << 18) + 4000, None), ("poly_matrix", 8, 10, 4, (1 << 18) + 5, None),
    ("cauchy", 8, 10, 4, 8 * 2048 * 8, 2048), ("cauchy", 8, 6, 3, 8 * 2048 * 3, 2048),
    ("cauchy", 16, 12, 4, 16 * 2048 * 2, 2048), ("cauchy", 8, 10, 4, 8 * 512 * 5, 512),
    ("cauchy", 8, 7, 5, 8 * 1024 * 3, 1024), ("cauchy", 16, 3, 2, 16 * 128 * 4, 128),
    ("cauchy", 8, 20, 4, 8 * 384 * 2, 384), ("cauchy", 8, 10, 4, 8 * 128 * 3, 128),
    ("cauchy", 8, 10, 4, 8 * 768 * 2, 768), ("poly_bitmatrix", 8, 10, 4, 8 * 640 * 2, 640),
    ("cauchy", 8, 10, 4, 8 * 512, 512), ("poly_bitmatrix", 8, 10, 4, 8 * 256 * 3, 256),
    ("poly_matrix", 8, 10, 4, 1 << 20, None), ("poly_matrix", 8, 10, 4, 65536 + 37, None),
    ("poly_matrix", 16, 12, 4, 100002, None), ("poly_matrix", 8, 7, 5, 50000, None),
    ("poly_bitmatrix", 8, 10, 4, 8 * 2048 * 8, 2048), ("poly_bitmatrix", 8, 6, 3, 8 * 1024 * 3, 1024),
    ("poly_bitmatrix", 16, 12, 4, 16 * 2048 * 2, 2048),
    # good Cauchy (GoodCRS): compiled codes, two-group decodes, runtime-P codes
    ("good_cauchy", 8, 10, 4, 8 * 2048 * 8, 2048), ("good_cauchy", 8, 6, 3, 8 * 2048 * 3, 2048),
    ("good_cauchy", 16, 12, 4, 16 * 2048 * 2, 2048), ("good_cauchy", 8, 10, 4, 8 * 512 * 5, 512),
    ("good_cauchy", 8, 7, 5, 8 * 1024 * 3, 1024), ("good_cauchy", 8, 20, 4, 8 * 384 * 2, 384),
    ("good_cauchy", 8, 12, 4, 8 * 2048 * 4, 2048), ("good_cauchy", 16, 3, 2, 16 * 128 * 4, 128),
]


@pytest.mark.parametrize("real,w,k,m,B,pkt", CASES)
def test_encode_bit_exact(rs, real, w, k, m, B, pkt):
    import torch
    code = rs.Code(k, m, w, real, packet_bytes=pkt)
    host = stripe(w, k, m, B)
    ref = host.copy()
    O.encode(real, w, k, m, ref, packet_bytes=pkt or 2048)
    buf, rows = device_blocks(host)
    buf[k:] = 0x5A
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    assert np.array_equal(to_host(buf, B), ref)


@pytest.mark.parametrize("read_mode", [0, 1])
@pytest.mark.parametrize("real,w,k,m,B,pkt", CASES)
def test_decode_bit_exact(rs, real, w, k, m, B, pkt, read_mode):
    import torch
    code = rs.Code(k, m, w, real, packet_bytes=pkt, read_mode=read_mode)
    host = stripe(w, k, m, B)
    O.encode(real, w, k, m, host, packet_bytes=pkt or 2048)
    n = k + m
    for s in range(m + 1):
        e = 1 + s % m
        er = inputs.erasure_pattern(inputs.stream_seed(2), s, n, e)
        bad = host.copy()
        bad[er] = 0xC3
        buf, rows = device_blocks(bad)
        code.decode(er, rows, B)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(buf, B), host), er
    assert code.poll_status() == 0


def test_generator_matrix_form_equals_lfsr(rs):
    """§6: the polynomial code through its generator matrix gives the LFSR's
    bytes (and the same decode)."""
    import torch
    k, m, w, B = 10, 4, 8, (1 << 20) + 48
    host = stripe(w, k, m, B)
    a_buf, a_rows = device_blocks(host)
    b_buf, b_rows = device_blocks(host)
    rs.Code(k, m, w, "poly").encode(a_rows[:k], a_rows[k:], B)
    rs.Code(k, m, w, "poly_matrix").encode(b_rows[:k], b_rows[k:], B)
    torch.cuda.synchronize()
    assert torch.equal(a_buf, b_buf)


def test_cauchy_block_size_must_fit_packets(rs):
    import torch
    code = rs.Code(10, 4, 8, "cauchy", packet_bytes=2048)
    t = torch.zeros((14, 16384 + 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.RSError):
        code.encode(list(t[:10]), list(t[10:]), 16384 + 16)
    with pytest.raises(rs.RSError):
        rs.rs_set_packet_bytes(code.handle, 100)


# Packet-layout tiles are runs of consumer_warps x 32 units (G words of each
# packet row); these shapes make tiles start inside a super-packet, span
# several, and end short at the block's end.  The GF(2^16) cases with 768-
# and 256-byte packets run the two-word-per-lane kernels (encodes, good
# Cauchy decode), 384-byte packets the one-word ones.
@pytest.mark.parametrize("warps", [1, 3, 5, 12, 16])
@pytest.mark.parametrize("real,w,k,m,pkt,nsp", [("cauchy", 8, 10, 4, 2048, 7), ("cauchy", 8, 10, 4, 256, 37),
                                                ("cauchy", 8, 10, 4, 768, 5), ("cauchy", 8, 7, 5, 640, 9),
                                                ("poly_bitmatrix", 8, 10, 4, 1024, 6),
                                                ("cauchy", 16, 12, 4, 384, 5), ("good_cauchy", 8, 10, 4, 768, 5),
                                                ("cauchy", 16, 12, 4, 768, 3), ("good_cauchy", 16, 12, 4, 768, 3),
                                                ("good_cauchy", 16, 12, 4, 256, 5)])
def test_packet_tiles_any_warp_count(rs, real, w, k, m, pkt, nsp, warps):
    import torch
    B = nsp * w * pkt
    code = rs.Code(k, m, w, real, packet_bytes=pkt)
    code.set_launch(warps, 4, 1)
    host = stripe(w, k, m, B, seed=11)
    ref = host.copy()
    O.encode(real, w, k, m, ref, packet_bytes=pkt)
    buf, rows = device_blocks(host)
    buf[k:] = 0x5A
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(buf, B), ref)
    n = k + m
    for s in range(3):
        er = inputs.erasure_pattern(inputs.stream_seed(3), s, n, m - s % 2)
        bad = ref.copy()
        bad[er] = 0xC3
        buf, rows = device_blocks(bad)
        code.decode(er, rows, B)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(buf, B), ref), er
    assert code.poll_status() == 0


def test_good_cauchy_has_fewer_ones_and_differs_from_cauchy(rs):
    """The good Cauchy code is a different code (other parity bytes) whose
    bit-matrix has fewer ones than the original's (the XOR count)."""
    import torch
    w, k, m, pkt = 8, 10, 4, 2048
    B = 8 * pkt * 4
    ones = lambda C: sum(O.bitmatrix_ones(w, int(x)) for x in C.ravel())
    assert ones(O.goodcauchy_matrix(w, k, m)) < ones(O.cauchy_matrix(w, k, m))
    host = stripe(w, k, m, B)
    a_buf, a_rows = device_blocks(host)
    b_buf, b_rows = device_blocks(host)
    rs.Code(k, m, w, "cauchy", packet_bytes=pkt).encode(a_rows[:k], a_rows[k:], B)
    rs.Code(k, m, w, "good_cauchy", packet_bytes=pkt).encode(b_rows[:k], b_rows[k:], B)
    torch.cuda.synchronize()
    assert torch.equal(a_buf[:k], b_buf[:k]) and not torch.equal(a_buf[k:], b_buf[k:])


@pytest.mark.parametrize("groups", [1, 2])
@pytest.mark.parametrize("real,w,k,m,B,pkt", [("poly", 8, 10, 4, (64 << 10) + 16, None),
                                              ("vandermonde", 8, 10, 4, (64 << 10) + 16, None),
                                              ("vandermonde", 8, 6, 3, 1 << 20, None),
                                              ("poly", 8, 10, 5, 100000, None),
                                              ("good_cauchy", 8, 10, 4, 8 * 2048 * 3, 2048),
                                              ("good_cauchy", 16, 12, 4, 16 * 2048, 2048)])
def test_forced_column_groups_match_oracle(rs, real, w, k, m, B, pkt, groups):
    """One or two 32-column groups per thread forced on either side of the
    block-size threshold give the oracle's bytes (encode, then a decode of
    m seeded erasures)."""
    import torch
    code = rs.Code(k, m, w, real, packet_bytes=pkt)
    code.set_launch(groups=groups)
    host = stripe(w, k, m, B, seed=13)
    ref = host.copy()
    O.encode(real, w, k, m, ref, packet_bytes=pkt or 2048)
    buf, rows = device_blocks(host)
    buf[k:] = 0x5A
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(buf, B), ref)
    er = inputs.erasure_pattern(inputs.stream_seed(5), groups, k + m, m)
    bad = ref.copy()
    bad[er] = 0xC3
    buf, rows = device_blocks(bad)
    code.decode(er, rows, B)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(buf, B), ref), er
    assert code.poll_status() == 0
