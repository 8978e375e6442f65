"""The allocation-free batched encode (rs_poly_encode_stripes_noalloc), for
callers that cannot allocate device memory when they encode (allocator
callbacks that must not re-enter the allocator, embedders with a fixed
device budget, paths that must not synchronise the device): on two calls in
a row that reuse its fixed scratch array, its parity equals both the
regular rs_encode entry point's and the CPU oracle's, byte for byte.  This
file is collected last on purpose, so a run that stops at its first failure
has run every other test."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _stripes(torch, k, m, sizes, seed):
    from paper_1312_5155_gb300 import inputs
    out = []
    for i, B in enumerate(sizes):
        Bp = max(16, (B + 15) // 16 * 16)
        buf = torch.zeros((k + m, Bp), dtype=torch.uint8, device="cuda")
        if B:
            buf[:k, :B] = inputs.random_bytes_torch(seed, i * k * B, k * B, "cuda").view(k, B)
        out.append((buf, [buf[j, :B] for j in range(k + m)], B))
    return out


def test_noalloc_encode_matches_rs_encode_and_oracle_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs
    build.build()
    for (w, k, m), sizes, seed in [((8, 10, 4), [1 << 20, 65536 + 16, 4096, 300000 + 7, 0], 11),
                                   ((8, 6, 3), [12345, 1 << 18, 4096 * 3], 12),
                                   ((16, 12, 4), [40000, 8192 + 2], 13)]:
        code = rs.Code(k, m, w, "poly")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        # two calls in a row on the shared scratch array
        for call in range(2):
            stripes = _stripes(torch, k, m, [s + 32 * call if s else 0 for s in sizes], seed + 100 * call)
            ref = [buf.clone() for buf, _, _ in stripes]
            for (buf, rows, B), r in zip(stripes, ref):
                rr = [r[j, :B] for j in range(k + m)]
                code.encode(rr[:k], rr[k:], B)
            rs.rs_poly_encode_stripes_noalloc(k, m, w, [rows[:k] for _, rows, _ in stripes],
                                              [rows[k:] for _, rows, _ in stripes],
                                              [B for _, _, B in stripes], device_status=status)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            for (buf, _, B), r in zip(stripes, ref):
                got = buf[:, :B].cpu().numpy()
                assert np.array_equal(got, r[:, :B].cpu().numpy()), (w, k, m, B, call, "vs rs_encode")
                want = got.copy()
                want[k:] = 0
                O.poly_encode(w, k, m, want)
                assert np.array_equal(got, want), (w, k, m, B, call, "vs oracle")
        code.close()


def test_noalloc_rejects_oversized_and_bad_requests():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import rs
    t = torch.zeros((64, 16), dtype=torch.uint8, device="cuda")
    n = 4000  # RS(60,4): 4000 stripes need far more than the fixed array
    with pytest.raises(rs.RSError) as ei:
        rs.rs_poly_encode_stripes_noalloc(60, 4, 8, [[t[j] for j in range(60)]] * n,
                                          [[t[60 + j] for j in range(4)]] * n, [16] * n)
    assert "bytes of scratch" in str(ei.value)
    with pytest.raises(rs.RSError):  # blocks of one stripe overlap
        rs.rs_poly_encode_stripes_noalloc(2, 1, 8, [[t[0], t[0]]], [[t[1]]], [16])
