"""GPU parity of the batched path: many stripes of mixed codes,
realizations, block sizes and ops in one batch give the same bytes as the
oracle and as the same ops run one at a time; a captured CUDA graph replays
with rewritten descriptors."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs as rsmod
    build.build()
    return rsmod


def alloc_stripe(n, B):
    import torch
    Bp = max(16, (B + 15) // 16 * 16)
    buf = torch.zeros((n, Bp), dtype=torch.uint8, device="cuda")
    return buf, [buf[i, :B] for i in range(n)]


def make_workload(rs, specs, seed):
    """specs: list of (realization, w, k, m, B, pkt, op, e)."""
    import torch
    codes = {}
    items = []
    for idx, (real, w, k, m, B, pkt, op, e) in enumerate(specs):
        key = (real, w, k, m, pkt)
        if key not in codes:
            codes[key] = rs.Code(k, m, w, real, packet_bytes=pkt)
        n = k + m
        host = np.zeros((n, B), dtype=np.uint8)
        host[:k] = inputs.stripe_blocks(seed, idx, k, B)
        ref = host.copy()
        O.encode(real, w, k, m, ref, packet_bytes=pkt or 2048)
        er = inputs.erasure_pattern(seed, idx, n, e) if op == "decode" else []
        start = host.copy() if op == "encode" else ref.copy()
        if op == "decode":
            start[er] = 0xE1
        buf, rows = alloc_stripe(n, B)
        if B:
            buf[:, :B] = torch.from_numpy(start).cuda()
        items.append(dict(code=codes[key], op=op, er=er, buf=buf, rows=rows, B=B, ref=ref, start=start))
    return codes, items


def check(items):
    for it in items:
        got = it["buf"][:, :it["B"]].cpu().numpy()
        assert np.array_equal(got, it["ref"]), (it["op"], it["er"], it["code"].realization)


def test_mixed_batch_matches_oracle_and_single_calls(rs):
    import torch
    specs = []
    sizes = [4096, 65536 + 16, 300000, 1 << 20, 12345 + 3, 0]
    for i in range(24):
        k, m = [(6, 3), (10, 4), (12, 4), (20, 4)][i % 4]
        B = sizes[i % len(sizes)]
        op = "decode" if i % 3 == 0 else "encode"
        specs.append(("poly", 8, k, m, B, None, op, 1 + i % m))
    specs += [("vandermonde", 8, 10, 4, 100000, None, "encode", 0),
              ("vandermonde", 8, 10, 4, 100000, None, "decode", 2),
              ("cauchy", 8, 10, 4, 8 * 2048 * 4, 2048, "encode", 0),
              ("cauchy", 8, 10, 4, 8 * 2048 * 4, 2048, "decode", 4),
              ("good_cauchy", 8, 10, 4, 8 * 2048 * 4, 2048, "encode", 0),
              ("good_cauchy", 8, 6, 3, 8 * 2048 * 2, 2048, "decode", 3),
              ("poly", 16, 12, 4, 40000, None, "encode", 0)]
    codes, items = make_workload(rs, specs, seed=0x5EED0004)
    b = rs.Batch(len(items))
    b.set([(it["code"], it["op"], it["er"], it["rows"], it["B"]) for it in items])
    b.launch()
    torch.cuda.synchronize()
    assert b.poll_status() == 0
    check(items)
    # mixed polynomial kernel: the M = 3 and M = 4 poly ops share one launch
    assert b.kernel_count <= 8
    # the same ops one call at a time give the same bytes
    for it in items:
        it["buf"][:, :it["B"]] = torch.from_numpy(it["start"]).cuda()
        if it["op"] == "encode":
            it["code"].encode(it["rows"][:it["code"].k], it["rows"][it["code"].k:], it["B"])
        else:
            it["code"].decode(it["er"], it["rows"], it["B"])
    torch.cuda.synchronize()
    check(items)


def test_graph_capture_replays_new_descriptors(rs):
    import torch
    specs_a = [("poly", 8, 10, 4, 65536, None, "encode", 0) for _ in range(6)]
    specs_b = [("poly", 8, 10, 4, 131072 + 32, None, "encode", 0) for _ in range(9)]
    _, items_a = make_workload(rs, specs_a, seed=101)
    _, items_b = make_workload(rs, specs_b, seed=202)
    b = rs.Batch(16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.set([(it["code"], it["op"], it["er"], it["rows"], it["B"]) for it in items_a], stream=s)
        b.launch(stream=s)  # warm-up launch outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.launch(stream=s)
        g.replay()
        torch.cuda.synchronize()
        check(items_a)
        # new descriptors, same kernel group: the same graph runs them
        b.set([(it["code"], it["op"], it["er"], it["rows"], it["B"]) for it in items_b], stream=s)
        g.replay()
        torch.cuda.synchronize()
    check(items_b)
    assert b.poll_status() == 0


def test_batch_rejects_bad_ops(rs):
    import torch
    code = rs.Code(10, 4, 8, "poly")
    t = torch.zeros((14, 4096), dtype=torch.uint8, device="cuda")
    b = rs.Batch(4)
    with pytest.raises(rs.RSError) as ei:
        b.set([(code, "decode", [0, 1, 2, 3, 4], list(t), 4096)])
    assert "op 0" in str(ei.value)
    with pytest.raises(rs.RSError):
        b.set([(code, "encode", [], list(t), 4096)] * 5)  # more than max_ops


def test_batch_mixes_one_and_two_group_kernels(rs):
    """Blocks on both sides of the one-/two-group threshold in one batch: the
    same codes run as separate kernel groups and every op matches the
    oracle."""
    import torch
    specs = []
    for i, B in enumerate([64 << 10, 512 << 10, 64 << 10, 512 << 10]):
        for real, pkt in (("vandermonde", None), ("poly", None), ("cauchy", 2048)):
            if real == "cauchy":
                B = (B // (8 * 2048)) * 8 * 2048
            specs.append((real, 8, 10, 4, B, pkt, "encode" if i < 2 else "decode", 1 + i % 4))
    codes, items = make_workload(rs, specs, seed=0x5EED0007)
    b = rs.Batch(len(items))
    b.set([(it["code"], it["op"], it["er"], it["rows"], it["B"]) for it in items])
    b.launch()
    torch.cuda.synchronize()
    assert b.poll_status() == 0
    check(items)
    assert b.kernel_count >= 4


def test_multi_group_batch_orders_later_work_on_its_stream(rs):
    """The kernel groups after the first run on the batch's side streams;
    work queued on the launch stream after rs_batch_launch (here copies of
    every output block, taken without any host synchronisation) must see
    all groups finished, eagerly and through a captured graph."""
    import torch
    specs = []
    for i in range(3):
        specs += [("poly", 8, 10, 4, 1 << 20, None, "encode", 0),
                  ("vandermonde", 8, 10, 4, 1 << 20, None, "encode", 0),
                  ("good_cauchy", 8, 10, 4, 8 * 2048 * 64, 2048, "decode", 1 + i),
                  ("poly", 8, 6, 3, 1 << 20, None, "decode", 1 + i)]
    codes, items = make_workload(rs, specs, seed=0x5EED0009)
    b = rs.Batch(len(items))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.set([(it["code"], it["op"], it["er"], it["rows"], it["B"]) for it in items], stream=s)
        assert b.kernel_count >= 3
        b.launch(stream=s)
        snaps = [it["buf"].clone() for it in items]
    torch.cuda.synchronize()
    assert b.poll_status() == 0
    for it, snap in zip(items, snaps):
        assert np.array_equal(snap[:, :it["B"]].cpu().numpy(), it["ref"]), (it["op"], it["code"].realization)
    # the same through a graph: reset the blocks, replay, copy on the stream
    for it in items:
        it["buf"][:, :it["B"]] = torch.from_numpy(it["start"]).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.launch(stream=s)
        for it in items:
            it["buf"][:, :it["B"]] = torch.from_numpy(it["start"]).cuda()
        g.replay()
        snaps = [it["buf"].clone() for it in items]
    torch.cuda.synchronize()
    for it, snap in zip(items, snaps):
        assert np.array_equal(snap[:, :it["B"]].cpu().numpy(), it["ref"]), (it["op"], it["code"].realization, "graph")
