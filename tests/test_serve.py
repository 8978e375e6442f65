"""Serving loop: host-side logic on CPU (arena, request generator), and on
the GPU that each request's result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_1312_5155_gb300 import serve


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(1 << 20)
    x = a.alloc(1000)
    y = a.alloc(5000)
    z = a.alloc(300)
    assert x == (0, 1024) and y[0] == 1024 and z[0] == 1024 + 5120
    assert a.alloc(1 << 20) is None
    a.release(*y)
    w = a.alloc(2048)
    assert w[0] == 1024  # first fit reuses the hole
    a.release(*x)
    a.release(*w)
    a.release(*z)
    assert a.free == [(0, 1 << 20)] and a.used == 0


def test_request_generator_statistics():
    reqs = serve.make_requests(0x5EED0005, rate=2000.0, seconds=2.0)
    n = len(reqs)
    assert 3400 < n < 4600  # Poisson(4000)
    B = np.array([r.block_bytes for r in reqs])
    assert np.all(B % 4096 == 0) and B.min() >= 4096 and B.max() <= 64 << 20
    assert 200 << 10 < np.median(B) < 320 << 10
    dec = [r for r in reqs if r.op == "decode"]
    assert 0.2 < len(dec) / n < 0.3
    for r in dec:
        assert 1 <= len(r.erasures) <= r.m and len(set(r.erasures)) == len(r.erasures)
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert {(r.k, r.m) for r in reqs} == set(serve.CODES)


def test_io_blocks():
    r = serve.Request(0, 0.0, 10, 4, "decode", 4096, erasures=[0, 11])
    read, write = serve.io_blocks(r)
    assert read == [1, 2, 3, 4, 5, 6, 7, 8, 9, 10] and write == [0, 11]
    r2 = serve.Request(1, 0.0, 6, 3, "encode", 4096)
    assert serve.io_blocks(r2) == ([0, 1, 2, 3, 4, 5], [6, 7, 8])


@pytest.mark.gpu
def test_served_results_equal_alone_results_and_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1312_5155_gb300 import build, inputs, rs
    build.build()
    reqs = serve.make_requests(0x5EED0005, rate=3000.0, seconds=0.05)
    assert len(reqs) > 50
    # distinct payload per request, encoded by the oracle
    payloads, expect = {}, {}
    for r in reqs:
        n, B = r.k + r.m, min(r.block_bytes, 256 << 10)
        r.block_bytes = B
        host = np.zeros((n, B), dtype=np.uint8)
        host[:r.k] = inputs.stripe_blocks(77, r.rid, r.k, B)
        O.poly_encode(8, r.k, r.m, host)
        _, d2h = serve.io_blocks(r)
        expect[r.rid] = host[d2h].copy()
        if r.op == "decode":
            host[r.erasures] = 0xBB
        payloads[r.rid] = torch.from_numpy(host).pin_memory()
    # in the mix: continuous batching over 3 streams, small budget so that
    # admission has to wait for memory
    results = serve.make_results(reqs)
    srv = serve.Server(64 << 20, streams=3, max_batch=16)
    srv.run(reqs, payloads, results)
    torch.cuda.synchronize()
    assert all(r.done >= r.arrival for r in reqs)
    for r in reqs:
        assert np.array_equal(results[r.rid].numpy(), expect[r.rid]), r.rid
    # alone: the serial path gives the same bytes
    codes = {c: rs.Code(c[0], c[1], 8, "poly") for c in serve.CODES}
    alone = serve.make_results(reqs)
    for r in reqs:
        r.arrival = 0.0
    serve.serial_run(reqs, payloads, alone, codes, torch.device("cuda"))
    for r in reqs:
        assert np.array_equal(alone[r.rid].numpy(), results[r.rid].numpy()), r.rid
    for s in srv.slots:
        assert s["batch"].poll_status() == 0


def test_add_range_merges_consecutive_rows():
    from paper_1312_5155_gb300.serve import _add_range
    d, s, n = [], [], []
    _add_range(d, s, n, 1000, 5000, 16)
    _add_range(d, s, n, 1016, 5016, 32)   # follows on: merged
    _add_range(d, s, n, 2000, 5048, 16)   # destination jumps: new range
    _add_range(d, s, n, 2016, 9000, 16)   # source jumps: new range
    _add_range(d, s, n, 2032, 9016, 16, join=False)  # another buffer: kept apart
    assert (d, s, n) == ([1000, 2000, 2016, 2032], [5000, 5048, 9000, 9016], [48, 16, 16, 16])
