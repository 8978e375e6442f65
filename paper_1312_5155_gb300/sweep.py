"""Throughput sweeps over the synthetic workloads of the polynomial
realization study (§5: random in-memory data, encode and decode of RS(k, m)
stripes; §5 Fig. 1-4: block size, k and m sweeps), run through the C ABI on
one GPU.

    python -m paper_1312_5155_gb300.sweep <name> [...]

Names:
  single_stripe  RS(10,4) poly, one stripe of 10 x 64 KiB: latency of one
            rs_encode / rs_decode call, and throughput of 1024 replicated
            stripes in one batched launch
  block_sizes  RS(6,3) and RS(10,4), GF(2^8), 1 GiB of data cut into stripes of
            B = 4 KiB * 2^i (i = 0..14), poly / Vandermonde / Cauchy / good
            Cauchy (P = min(2 KiB, B/8)): batched encode, then batched decode
            with m seeded erasures per stripe
  gf16_blocks  RS(12,4) GF(2^16) little-endian, 42 stripes of 4 MiB blocks:
            poly, Cauchy and good Cauchy encode, decode with e = 1..4
  mixed_batch  4096 stripes, (k, m) uniform over (6,3) (10,4) (12,4) (20,4),
            B log-uniform on [4 KiB, 8 MiB] (multiples of 4 KiB), 30 %
            decodes with e uniform in 1..m, poly: one batched launch set vs a
            loop of per-stripe rs_encode / rs_decode calls
  kmsweep   (k, 4) for k = 2..20 and (10, m) for m = 2..6, GF(2^8), 1 MiB
            blocks, 1 GiB of data, poly / Vandermonde / Cauchy / good Cauchy
  polyforms the polynomial code as LFSR, through its generator matrix and
            through that matrix's bit-matrix (packets), RS(10,4), RS(12,4),
            RS(6,3), 1 MiB blocks
  profile   one small case for ncu (--op, --code k:m, --w, --block, --stripes;
            default RS(12,4) GF(2^16) 4 MiB x 16 stripes)

Every line printed is one JSON object.  Bytes are algorithmic: encode
(k + m) B, decode (k + e) B per stripe (min-read); "user_gbs" is k B / t.
Inputs are the seeded SplitMix64 streams of inputs.py; times are CUDA events
on the launching stream after warm-up, median of the timed repetitions.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics

from . import autotune, inputs, rs

GIB = 1 << 30
# launch shapes tried per case (consumer warps, ring depth, CTAs per SM): the
# ones the bench's autotuner picks for these kernels
SHAPES = [(16, 8, 1), (16, 12, 1), (12, 4, 1), (12, 6, 1), (8, 12, 2), (8, 8, 2)]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    return torch


def _time(fn, reps=10, warm=3):
    torch = _torch()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _fill(buf, seed, k, B, stripes):
    """Data blocks of stripes 0..stripes-1 of a workload's byte stream."""
    torch = _torch()
    per = max(1, (256 << 20) // max(1, k * B))
    for s0 in range(0, stripes, per):
        s1 = min(stripes, s0 + per)
        buf[s0:s1, :k] = inputs.random_bytes_torch(seed, s0 * k * B, (s1 - s0) * k * B, "cuda").view(s1 - s0, k, B)
    torch.cuda.synchronize()


def _packet(real, w, B):
    if real not in rs.PACKET_REALIZATIONS:
        return None
    return min(2048, B // w)


def _batch_pair(real, w, k, m, B, stripes, seed, e, tune=True, tag=""):
    """Time batched encode and decode of `stripes` stripes; returns a dict."""
    torch = _torch()
    n = k + m
    buf = torch.empty((stripes, n, B), dtype=torch.uint8, device="cuda")
    _fill(buf, seed, k, B, stripes)
    code = rs.Code(k, m, w, real, packet_bytes=_packet(real, w, B))
    base = buf.data_ptr()
    rows = [[base + (s * n + j) * B for j in range(n)] for s in range(stripes)]  # device pointers
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    enc_ops = [(code, "encode", [], rows[s], B) for s in range(stripes)]
    dec_ops = [(code, "decode", inputs.erasure_pattern(seed, s, n, e), rows[s], B) for s in range(stripes)]
    out = {}
    for op, ops in (("encode", enc_ops), ("decode", dec_ops)):
        b = rs.Batch(stripes)
        b.set(ops)
        if tune:
            key = autotune.make_key(f"sweep{tag}{stripes}-{op}", real, k, m, w, B, sms)
            # small blocks fill only narrow tiles: try the tuner's whole list
            shape, _ = autotune.tune_batch(b, ops, key=key,
                                           candidates=autotune.CANDIDATES if B <= (16 << 10) else SHAPES)
        else:
            shape = (8, 16, 1)
            b.set_launch(*shape)
            b.set(ops)
        ms = _time(b.launch)
        if b.poll_status() != 0:
            raise RuntimeError(f"device status set ({real} {op})")
        nbytes = stripes * ((k + m) if op == "encode" else (k + e)) * B
        out[op] = {"ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
                   "user_gbs": round(stripes * k * B / ms / 1e6, 1), "shape": list(shape)}
        b.close()
    del buf
    torch.cuda.empty_cache()
    return out


def single_stripe():
    torch = _torch()
    k, m, w, B = 10, 4, 8, 64 << 10
    seed = inputs.workload_seed("single_stripe")
    n = k + m
    buf = torch.empty((n, B), dtype=torch.uint8, device="cuda")
    _fill(buf.view(1, n, B), seed, k, B, 1)
    code = rs.Code(k, m, w, "poly")
    rows = list(buf)
    er = inputs.erasure_pattern(seed, 0, n, m)
    enc = lambda: code.encode(rows[:k], rows[k:], B)  # noqa: E731
    dec = lambda: code.decode(er, rows, B)  # noqa: E731
    lat_e = _time(enc, reps=50)
    lat_d = _time(dec, reps=50)
    # the device side of one call alone: the same call captured in a CUDA
    # graph and replayed (no Python or ctypes work between the events)
    g_e, g_d = _graph_of(enc), _graph_of(dec)
    dev_e = _time(g_e.replay, reps=50)
    dev_d = _time(g_d.replay, reps=50)
    print(json.dumps({"workload": "single_stripe", "what": "one stripe, one call", "encode_us": round(lat_e * 1e3, 1),
                      "decode_us": round(lat_d * 1e3, 1), "graph_replay_encode_us": round(dev_e * 1e3, 1),
                      "graph_replay_decode_us": round(dev_d * 1e3, 1)}), flush=True)
    del buf
    r = _batch_pair("poly", w, k, m, B, 1024, seed, m, tag="c1-")
    print(json.dumps({"workload": "single_stripe", "what": "1024 replicated stripes, batched", **r}), flush=True)


def block_sizes(blocks=None, codes=((6, 3), (10, 4)), reals=("poly", "vandermonde", "cauchy", "good_cauchy")):
    seed = inputs.workload_seed("block_sizes")
    for (k, m) in codes:
        for i in (blocks if blocks is not None else range(15)):
            B = 4096 << i
            stripes = max(1, GIB // (k * B))
            for real in reals:
                r = _batch_pair(real, 8, k, m, B, stripes, seed, m, tag="c2-")
                print(json.dumps({"workload": "block_sizes", "k": k, "m": m, "B": B, "stripes": stripes, "realization": real,
                                  "packet_bytes": _packet(real, 8, B), **r}), flush=True)


def gf16_blocks(erasures=(1, 2, 3, 4), emit=True):
    """Config 3: RS(12,4) over GF(2^16), 4 MiB blocks, 42 stripes (2.8 GB),
    batched encode and decode with each erasure count, per realization.
    Returns the result dicts (and prints each as a JSON line if `emit`)."""
    torch = _torch()
    k, m, w, B, stripes = 12, 4, 16, 4 << 20, 42
    seed = inputs.workload_seed("gf16_blocks")
    n = k + m
    results = []
    for real in ("poly", "cauchy", "good_cauchy"):
        buf = torch.empty((stripes, n, B), dtype=torch.uint8, device="cuda")
        _fill(buf, seed, k, B, stripes)
        code = rs.Code(k, m, w, real, packet_bytes=_packet(real, w, B))
        rows = [list(buf[s]) for s in range(stripes)]
        res = {}
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        b = rs.Batch(stripes)
        ops = [(code, "encode", [], rows[s], B) for s in range(stripes)]
        shape, _ = autotune.tune_batch(b, ops, key=autotune.make_key(f"gf16-{stripes}-encode", real, k, m, w, B, sms))
        ms = _time(b.launch)
        res["encode"] = {"ms": round(ms, 4), "gbs": round(stripes * n * B / ms / 1e6, 1), "shape": list(shape)}
        for e in erasures:
            d = rs.Batch(stripes)
            ops = [(code, "decode", inputs.erasure_pattern(seed, s, n, e), rows[s], B) for s in range(stripes)]
            autotune.tune_batch(d, ops, key=autotune.make_key(f"gf16-{stripes}-decode{e}", real, k, m, w, B, sms))
            ms = _time(d.launch)
            if d.poll_status() != 0:
                raise RuntimeError("device status set")
            res[f"decode_e{e}"] = {"ms": round(ms, 4), "gbs": round(stripes * (k + e) * B / ms / 1e6, 1)}
            d.close()
        b.close()
        results.append({"workload": "gf16_blocks", "realization": real, "w": w, "B": B, "stripes": stripes, **res})
        if emit:
            print(json.dumps(results[-1]), flush=True)
        del buf
        torch.cuda.empty_cache()
    return results


def _graph_of(launch):
    """A CUDA graph holding one call of `launch` (captured on a side stream
    after a warm-up call outside the capture)."""
    torch = _torch()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        launch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            launch()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return g


def _percentile(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


def profile(op="good_cauchy_encode", k=12, m=4, w=16, B=4 << 20, stripes=16, launches=3):
    """One small case for ncu: `stripes` stripes of RS(k, m) over GF(2^w)
    with B-byte blocks (the default, 16 stripes of RS(12,4) GF(2^16) 4 MiB,
    is 1 GiB, larger than L2), one realization and op ("<realization>_encode"
    or "<realization>_decode", m erasures), the autotuned launch shape (tuned
    in the run before ncu's, then read from the tuner's cache), an encode
    that makes the parity valid, then `launches` launches of the op."""
    torch = _torch()
    real, kind = op.rsplit("_", 1)
    tag = "gf16" if (k, m, w, B) == (12, 4, 16, 4 << 20) else f"prof{k}-{m}-{w}-{B}"
    seed = inputs.workload_seed("gf16_blocks" if w == 16 else "block_sizes")
    n = k + m
    buf = torch.empty((stripes, n, B), dtype=torch.uint8, device="cuda")
    _fill(buf, seed, k, B, stripes)
    code = rs.Code(k, m, w, real, packet_bytes=_packet(real, w, B))
    rows = [list(buf[s]) for s in range(stripes)]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    enc_ops = [(code, "encode", [], rows[s], B) for s in range(stripes)]
    enc = rs.Batch(stripes)
    enc.set(enc_ops)
    enc.launch()
    if kind == "encode":
        b, ops = enc, enc_ops
    else:
        b = rs.Batch(stripes)
        ops = [(code, "decode", inputs.erasure_pattern(seed, s, n, m), rows[s], B) for s in range(stripes)]
        b.set(ops)
    shape, _ = autotune.tune_batch(b, ops, key=autotune.make_key(f"{tag}-{stripes}-{kind}", real, k, m, w, B, sms),
                                   candidates=autotune.CANDIDATES)
    torch.cuda.synchronize()
    for _ in range(launches):
        b.launch()
    torch.cuda.synchronize()
    if b.poll_status() != 0:
        raise SystemExit("device status word set")
    print(json.dumps({"profile": op, "k": k, "m": m, "w": w, "B": B, "stripes": stripes, "shape": list(shape)}),
          flush=True)


def mixed_batch(stripes=4096, reps=5, emit=True):
    """Config-4 batch: all stripes submitted at once.  Batched form = the
    persistent launches of one rs_batch, captured once in a CUDA graph and
    replayed; per-stripe form = one rs_encode / rs_decode call per stripe on
    the same stream.  Per-op latency = completion time of the op measured
    from the submission of the whole batch (batched: the end of the graph
    replay, which completes every op; loop: a CUDA event after each call)."""
    torch = _torch()
    seed = inputs.workload_seed("mixed_batch")
    shapes = inputs.mixed_batch_shapes(seed, stripes)
    total = sum((k + m) * B for k, m, B, _, _ in shapes)
    arena = torch.empty(total, dtype=torch.uint8, device="cuda")
    code = {c: rs.Code(c[0], c[1], 8, "poly") for c in inputs.MIXED_CODES}
    views = []
    for s, (k, m, B, e, off) in enumerate(shapes):
        v = arena[off:off + (k + m) * B].view(k + m, B)
        v[:k] = inputs.random_bytes_torch(seed, off, k * B, "cuda").view(k, B)
        views.append(v)
    torch.cuda.synchronize()
    # valid parity first so the decodes rebuild real codewords
    enc_all = rs.Batch(stripes)
    enc_all.set([(code[(k, m)], "encode", [], list(views[s]), B) for s, (k, m, B, e, _) in enumerate(shapes)])
    enc_all.launch()
    torch.cuda.synchronize()
    ops = mixed_batch_ops(seed, shapes, views, code)
    nbytes = sum((k + m) * B if not e else (k + e) * B for k, m, B, e, _ in shapes)
    b = rs.Batch(stripes)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    shape, _ = autotune.tune_batch(b, ops, key=autotune.make_key(f"mixed_batch-{stripes}", "poly-mixed", 0, 0, 8,
                                                                  1 << 20, sms))
    ms_batch = _time(b.launch, reps=reps, warm=2)
    g = _graph_of(b.launch)
    ms_graph = _time(g.replay, reps=reps, warm=2)
    if b.poll_status() != 0:
        raise RuntimeError("device status set")
    # the same ops as a loop of per-stripe calls on one stream
    calls = []
    for c, op, er, rows, B in ops:
        if op == "encode":
            calls.append((c.encode, (rows[:c.k], rows[c.k:], B)))
        else:
            calls.append((c.decode, (er, rows, B)))

    def loop(evs=None):
        for i, (f, a) in enumerate(calls):
            f(*a)
            if evs is not None:
                evs[i].record()

    ms_loop = _time(loop, reps=reps, warm=1)
    t0 = torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in calls]
    t0.record()
    loop(evs)
    torch.cuda.synchronize()
    lat_loop = [t0.elapsed_time(e) for e in evs]
    lat_graph = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        lat_graph.append(e0.elapsed_time(e1))
    res = {"workload": "mixed_batch", "stripes": stripes, "bytes": nbytes,
                      "gib_resident": round(total / GIB, 2), "decodes": sum(1 for x in shapes if x[3]),
                      "kernel_launches_batched": b.kernel_count, "launch_shape": list(shape),
                      "batched": {"ms": round(ms_batch, 3), "gbs": round(nbytes / ms_batch / 1e6, 1)},
                      "graph_replay": {"ms": round(ms_graph, 3), "gbs": round(nbytes / ms_graph / 1e6, 1),
                                       "op_latency_p50_ms": round(statistics.median(lat_graph), 3),
                                       "op_latency_p99_ms": round(max(lat_graph), 3)},
                      "per_stripe_loop": {"ms": round(ms_loop, 3), "gbs": round(nbytes / ms_loop / 1e6, 1),
                                          "op_latency_p50_ms": round(_percentile(lat_loop, 0.5), 3),
                                          "op_latency_p99_ms": round(_percentile(lat_loop, 0.99), 3)}}
    if emit:
        print(json.dumps(res), flush=True)
    b.close()
    enc_all.close()
    return res


def mixed_batch_ops(seed, shapes, views, code):
    """The batch's ops: stripe s is decoded (erasure pattern of stripe s, e
    blocks) when its shape has e > 0, else encoded."""
    ops = []
    for s, (k, m, B, e, _) in enumerate(shapes):
        if e:
            ops.append((code[(k, m)], "decode", inputs.erasure_pattern(seed, s, k + m, e), list(views[s]), B))
        else:
            ops.append((code[(k, m)], "encode", [], list(views[s]), B))
    return ops


def kmsweep(points=None):
    """§5.2 Fig. 3 and 4 on the GPU.  Every matrix realization runs a
    compiled generator at every point when the library was built with
    RSGB_BUILD_KM_CODES=1; `compiled_generator` in each line reads the same
    variable, so set it for the sweep as for the build."""
    from . import build
    compiled = set(build.fixed_codes())
    seed = inputs.workload_seed("block_sizes")
    B = 1 << 20
    for (k, m) in points or [(k, 4) for k in range(2, 21)] + [(10, m) for m in (2, 3, 5, 6)]:
        stripes = max(1, GIB // (k * B))
        for real in ("poly", "vandermonde", "cauchy", "good_cauchy"):
            r = _batch_pair(real, 8, k, m, B, stripes, seed, m, tag="km-")
            print(json.dumps({"sweep": "km", "k": k, "m": m, "B": B, "stripes": stripes, "realization": real,
                              "compiled_generator": real == "poly" or (8, k, m) in compiled, **r}), flush=True)


def polyforms():
    """The three device forms of the polynomial code (§3 LFSR; §6's open
    questions: its generator matrix in the symbol layout and that matrix's
    bit-matrix projection over packets), RS(10,4) and RS(12,4) over 1 GiB
    of 1 MiB blocks."""
    seed = inputs.workload_seed("block_sizes")
    B = 1 << 20
    for (k, m) in ((10, 4), (12, 4), (6, 3)):
        stripes = max(1, GIB // (k * B))
        for real in ("poly", "poly_matrix", "poly_bitmatrix"):
            r = _batch_pair(real, 8, k, m, B, stripes, seed, m, tag="pf-")
            print(json.dumps({"sweep": "polyforms", "k": k, "m": m, "B": B, "stripes": stripes,
                              "realization": real, **r}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("name", nargs="+", choices=["single_stripe", "block_sizes", "gf16_blocks", "mixed_batch", "kmsweep",
                                                     "polyforms", "profile"])
    ap.add_argument("--op", default="good_cauchy_encode", help="profile: <realization>_encode|_decode")
    ap.add_argument("--code", default="12:4", help="profile: k:m")
    ap.add_argument("--w", type=int, default=16, help="profile: field width")
    ap.add_argument("--block", type=int, default=4 << 20, help="profile: block bytes")
    ap.add_argument("--stripes", type=int, default=16, help="profile: stripes")
    ap.add_argument("--blocks", default=None, help="block_sizes: comma-separated exponents i (B = 4 KiB * 2^i)")
    ap.add_argument("--codes", default=None, help="kmsweep: comma-separated k:m points (default: the whole study)")
    a = ap.parse_args()
    for name in a.name:
        if name == "block_sizes" and a.blocks:
            block_sizes(blocks=[int(x) for x in a.blocks.split(",")])
        elif name == "profile":
            pk, pm = (int(x) for x in a.code.split(":"))
            profile(a.op, pk, pm, a.w, a.block, a.stripes)
        elif name == "kmsweep" and a.codes:
            kmsweep(points=[tuple(int(v) for v in x.split(":")) for x in a.codes.split(",")])
        else:
            globals()[name]()


if __name__ == "__main__":
    main()
