"""GPU parity: polynomial realization through the C ABI vs the CPU oracle.

Bit-exact comparison on seeded inputs (tolerance: 0 differing bytes).
Sizes span several tiles and ragged tails; full-size configurations are
checked on sampled stripes.
"""
import itertools

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


def encode_case(rs, w, k, m, B, seed=1, stripe=0, launch=None):
    import torch
    code = rs.Code(k, m, w, "poly")
    if launch:
        code.set_launch(*launch)
    host = np.zeros((k + m, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(inputs.stream_seed(seed), stripe, k, B)
    ref = host.copy()
    O.poly_encode(w, k, m, ref)
    buf, rows = device_blocks(host)
    if B:
        buf[k:, :B] = 0xA5
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    got = to_host(buf, B)
    return got, ref


ENC = [(8, 10, 4, 16), (8, 10, 4, 1000), (8, 10, 4, 65536), (8, 10, 4, 65536 + 37),
       (8, 10, 4, 1 << 20), (8, 6, 3, 4096), (8, 20, 4, 300000), (8, 12, 4, 12345),
       (16, 12, 4, 2), (16, 12, 4, 8192), (16, 12, 4, 100002), (16, 6, 3, 4096 + 18)]


@pytest.mark.parametrize("w,k,m,B", ENC)
def test_encode_bit_exact(rs, w, k, m, B):
    got, ref = encode_case(rs, w, k, m, B)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("w,m", [(8, m) for m in range(1, 9)] + [(16, m) for m in range(1, 5)])
def test_encode_every_m(rs, w, m):
    k = 10 if m <= 6 else 8
    got, ref = encode_case(rs, w, k, m, 8192 + 64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("launch", [(1, 2, 1), (4, 4, 2), (16, 8, 1), (8, 32, 1), (2, 3, 4)])
def test_encode_launch_shapes(rs, launch):
    got, ref = encode_case(rs, 8, 10, 4, 200000 + 48, launch=launch)
    assert np.array_equal(got, ref)


def test_empty_block_is_noop(rs):
    import torch
    code = rs.Code(10, 4, 8, "poly")
    t = torch.full((14, 16), 7, dtype=torch.uint8, device="cuda")
    code.encode(list(t[:10]), list(t[10:]), 0)
    code.decode([0, 1], list(t), 0)
    torch.cuda.synchronize()
    assert int(t.sum()) == 7 * 14 * 16


def decode_case(rs, w, k, m, B, er, read_mode, seed=2, stripe=0):
    import torch
    code = rs.Code(k, m, w, "poly", read_mode=read_mode)
    n = k + m
    host = np.zeros((n, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(inputs.stream_seed(seed), stripe, k, B)
    O.poly_encode(w, k, m, host)
    ref = host.copy()
    ref[er] = 0
    O.poly_decode(w, k, m, er, ref)
    bad = host.copy()
    bad[er] = 0x3C
    buf, rows = device_blocks(bad)
    code.decode(er, rows, B)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    return to_host(buf, B), ref


@pytest.mark.parametrize("read_mode", [0, 1])
@pytest.mark.parametrize("w,k,m,B", [(8, 10, 4, 65536 + 16), (8, 6, 3, 5000), (16, 12, 4, 40002),
                                     (8, 20, 4, 100000), (8, 10, 8, 9000), (8, 10, 4, (1 << 18) + 37),
                                     (8, 6, 3, 300001), (8, 12, 4, 1 << 19), (8, 10, 5, (1 << 18) + 48),
                                     (8, 10, 6, 300000 + 16)])
def test_decode_seeded_patterns(rs, w, k, m, B, read_mode):
    n = k + m
    seed = inputs.stream_seed(2)
    for stripe in range(2 * m):
        e = 1 + stripe % m
        er = inputs.erasure_pattern(seed, stripe, n, e)
        got, ref = decode_case(rs, w, k, m, B, er, read_mode, stripe=stripe)
        assert np.array_equal(got, ref), er


def test_decode_all_patterns_rs_6_3(rs):
    import torch
    w, k, m, B = 8, 6, 3, 3000
    n = k + m
    code = rs.Code(k, m, w, "poly")
    host = np.zeros((n, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(5, 0, k, B)
    O.poly_encode(w, k, m, host)
    buf, rows = device_blocks(host)
    for e in range(1, m + 1):
        for er in itertools.combinations(range(n), e):
            buf[list(er), :B] = 0
            code.decode(list(er), rows, B)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(buf, B), host), er


def test_single_stripe_rs_10_4_64k(rs):
    """The single-stripe workload: RS(10,4), GF(2^8), one stripe of 10 x
    64 KiB; encode, then erase 4 seeded blocks of 14 and decode."""
    import torch
    w, k, m, B = 8, 10, 4, 65536
    seed = inputs.workload_seed("single_stripe")
    got, ref = encode_case(rs, w, k, m, B, seed=1)
    assert np.array_equal(got, ref)
    er = inputs.erasure_pattern(seed, 0, k + m, 4)
    code = rs.Code(k, m, w, "poly")
    bad = ref.copy()
    bad[er] = 0
    buf, rows = device_blocks(bad)
    code.decode(er, rows, B)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(buf, B), ref)


def test_argument_errors(rs):
    import torch
    code = rs.Code(10, 4, 8, "poly")
    t = torch.zeros((15, 4096), dtype=torch.uint8, device="cuda")
    rows = list(t[:14])
    with pytest.raises(rs.RSError) as ei:
        code.decode([0, 1, 2, 3, 4], rows, 4096)
    assert ei.value.status == 2
    with pytest.raises(rs.RSError):
        code.decode([1, 1], rows, 4096)
    with pytest.raises(rs.RSError):
        code.decode([14], rows, 4096)
    mis = [t.view(-1)[1 + 4096 * i:4096 * (i + 1)] for i in range(14)]
    with pytest.raises(rs.RSError) as ei:
        code.encode(mis[:10], mis[10:], 4000)
    assert "aligned" in str(ei.value)
    with pytest.raises(rs.RSError) as ei:
        code.encode(rows[:10], [rows[0]] + rows[11:], 4096)
    assert "overlap" in str(ei.value)
    c16 = rs.Code(12, 4, 16, "poly")
    t16 = torch.zeros((16, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.RSError):
        c16.encode(list(t16[:12]), list(t16[12:]), 4095)
