"""GPU parity at full size for the configurations that are too large for the
oracle to redo whole: the 4096-stripe mixed batch (about 67 GiB resident,
codes (6,3) (10,4) (12,4) (20,4), blocks of 4 KiB - 8 MiB, 30 % decodes) and
the extremes of the block-size and GF(2^16) studies (one RS(10,4) stripe of
64 MiB blocks in every realization; RS(12,4) over GF(2^16) with 4 MiB blocks
and 1..4 erasures in every realization).

The oracle checks seeded samples: in the symbol layout every byte offset
(GF(2^8)) or 16-bit word (GF(2^16)) is a codeword of its own, so a window of
columns of all n blocks is checked against the oracle's encode of the same
window of the data; in the packet layout whole super-packets are the
independent units.  The mixed batch is checked on the first and last 64 KiB
of every block of every stripe and on 64 whole stripes.  Every check runs
after the decode, on all n blocks: rebuilt blocks must equal the original
data or parity, the others must hold the encode's parity."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs

pytestmark = pytest.mark.gpu

WINDOW = 64 << 10


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs as rsmod
    build.build()
    return rsmod


def _windows(B, align=1):
    """Column windows (col0, ncols): the first and last WINDOW bytes of a
    block (the whole block when it is at most 2 * WINDOW)."""
    if B <= 2 * WINDOW:
        return [(0, B)]
    last = (B - WINDOW) // align * align
    return [(0, WINDOW), (last, B - last)]


def _expected(real, w, k, m, data_window, P=2048):
    ref = np.zeros((k + m, data_window.shape[1]), dtype=np.uint8)
    ref[:k] = data_window
    O.encode(real, w, k, m, ref, packet_bytes=P)
    return ref


def test_mixed_batch_4096_stripes_sampled(rs):
    import torch
    from paper_1312_5155_gb300 import sweep
    seed = inputs.workload_seed("mixed_batch")
    shapes = inputs.mixed_batch_shapes(seed, 4096)
    total = sum((k + m) * B for k, m, B, _, _ in shapes)
    arena = torch.empty(total, dtype=torch.uint8, device="cuda")
    code = {c: rs.Code(c[0], c[1], 8, "poly") for c in inputs.MIXED_CODES}
    views = []
    for k, m, B, e, off in shapes:
        v = arena[off:off + (k + m) * B].view(k + m, B)
        v[:k] = inputs.random_bytes_torch(seed, off, k * B, "cuda").view(k, B)
        v[k:] = 0x3C  # parity not yet written
        views.append(v)
    # every stripe encoded in one batch, then the mixed batch: encodes
    # (parity recomputed in place) and decodes of stripes whose erased
    # blocks were overwritten
    enc = rs.Batch(len(shapes))
    enc.set([(code[(k, m)], "encode", [], list(views[s]), B) for s, (k, m, B, e, _) in enumerate(shapes)])
    enc.launch()
    torch.cuda.synchronize()
    assert enc.poll_status() == 0
    ops = sweep.mixed_batch_ops(seed, shapes, views, code)
    for s, (c, op, er, rows, B) in enumerate(ops):
        for b in er:
            views[s][b].fill_(0xE1)
    mixed = rs.Batch(len(ops))
    mixed.set(ops)
    mixed.launch()
    torch.cuda.synchronize()
    assert mixed.poll_status() == 0
    assert mixed.kernel_count >= 1

    rng = np.random.default_rng(0x5EED4)
    whole = set(int(x) for x in rng.choice(len(shapes), 64, replace=False))

    def check(s):
        k, m, B, e, off = shapes[s]
        wins = [(0, B)] if s in whole else _windows(B)
        for col0, n in wins:
            data = np.stack([inputs.random_bytes(seed, off + j * B + col0, n) for j in range(k)])
            ref = _expected("poly", 8, k, m, data)
            got = views[s][:, col0:col0 + n].cpu().numpy()
            if not np.array_equal(got, ref):
                bad = np.argwhere(got != ref)[0]
                return f"stripe {s} {(k, m, B, e)} window {col0}+{n}: first mismatch block {bad[0]} col {bad[1]}"
        return None

    with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 4)) as ex:
        errs = [r for r in ex.map(check, range(len(shapes))) if r]
    assert not errs, errs[:5]


@pytest.mark.parametrize("real", ["poly", "vandermonde", "cauchy", "poly_matrix", "poly_bitmatrix", "good_cauchy"])
def test_rs10_4_64mib_blocks_sampled(rs, real):
    import torch
    k, m, w, B, P = 10, 4, 8, 64 << 20, 2048
    seed = inputs.workload_seed("block_sizes")
    n = k + m
    code = rs.Code(k, m, w, real, packet_bytes=P if real in rs.PACKET_REALIZATIONS else None)
    buf = torch.empty((n, B), dtype=torch.uint8, device="cuda")
    buf[:k] = inputs.random_bytes_torch(seed, 0, k * B, "cuda").view(k, B)
    rows = list(buf)
    code.encode(rows[:k], rows[k:], B)
    er = inputs.erasure_pattern(seed, 0, n, m)
    buf[er] = 0xE1
    code.decode(er, rows, B)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    rng = np.random.default_rng(0x64)
    if real in rs.PACKET_REALIZATIONS:
        sp = w * P  # super-packets are the independent units of the packet layout
        n_sp = B // sp
        picks = sorted({0, n_sp - 1} | set(int(x) for x in rng.choice(n_sp, 6, replace=False)))
        wins = [(i * sp, sp) for i in picks]
    else:
        wins = _windows(B) + [(int(c), 1) for c in rng.choice(B, 256, replace=False)]
    for col0, nc in wins:
        data = np.stack([inputs.random_bytes(seed, j * B + col0, nc) for j in range(k)])
        ref = _expected(real, w, k, m, data, P)
        got = buf[:, col0:col0 + nc].cpu().numpy()
        assert np.array_equal(got, ref), (real, col0, nc, er)


@pytest.mark.parametrize("real", ["poly", "vandermonde", "cauchy", "good_cauchy"])
def test_rs12_4_gf16_4mib_blocks_sampled(rs, real):
    import torch
    k, m, w, B, P = 12, 4, 16, 4 << 20, 2048
    seed = inputs.workload_seed("gf16_blocks")
    n = k + m
    stripes = 4
    code = rs.Code(k, m, w, real, packet_bytes=P if real in rs.PACKET_REALIZATIONS else None)
    buf = torch.empty((stripes, n, B), dtype=torch.uint8, device="cuda")
    buf[:, :k] = inputs.random_bytes_torch(seed, 0, stripes * k * B, "cuda").view(stripes, k, B)
    ref_stripes = []
    for s in range(stripes):
        rows = list(buf[s])
        code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0x16)
    for s in range(stripes):
        e = 1 + s  # 1..4 erasures
        er = inputs.erasure_pattern(seed, s, n, e)
        buf[s, er] = 0xE1
        code.decode(er, list(buf[s]), B)
        ref_stripes.append(er)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    for s in range(stripes):
        if real in rs.PACKET_REALIZATIONS:
            sp = w * P
            n_sp = B // sp
            picks = sorted({0, n_sp - 1} | set(int(x) for x in rng.choice(n_sp, 4, replace=False)))
            wins = [(i * sp, sp) for i in picks]
        else:
            wins = _windows(B, align=2) + [(2 * int(c), 2) for c in rng.choice(B // 2, 128, replace=False)]
        for col0, nc in wins:
            data = np.stack([inputs.random_bytes(seed, (s * k + j) * B + col0, nc) for j in range(k)])
            ref = _expected(real, w, k, m, data, P)
            got = buf[s, :, col0:col0 + nc].cpu().numpy()
            assert np.array_equal(got, ref), (real, s, col0, nc, ref_stripes[s])
