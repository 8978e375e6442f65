#!/usr/bin/env python
"""Encode/decode throughput of the GB300 Reed-Solomon library.

Workload (one step), from the RS(10,4) GF(2^8) part of the 1 GiB
block-size study: 1 GiB of uniform-random data cut into stripes of
10 blocks x 1 MiB (102 stripes).  For each realization -- polynomial (§3),
Vandermonde matrix (§2.2), Cauchy bit-matrix with 2 KiB packets (§2.3) and
its "good" matrix (GoodCRS, §2.3 / §5.1) -- a step encodes all 102 stripes
(one batched persistent launch), then decodes all 102 stripes with m = 4
seeded erasures each (one launch; min-read: the first k survivors are
read).  Inputs (4 x 1.4 GiB) are resident in HBM and larger than L2 when
the timed region starts.

value = algorithmic bytes / time: a stripe encode moves (k+m)*B bytes
(read k blocks, write m), a 4-erasure min-read decode (k+4)*B.
`user_gbs` counts data bytes k*B per stripe-op.  N > 1 (torchrun): every
rank runs the same per-GPU workload on its own stripes (weak scaling, no
collective on the data path); value = bytes of all ranks / max rank time.
The line also carries `e2e` (the step through the C ABI with its host
transfers), `serve` (request latency p50 / p99 of the continuous-batching
server at half its saturation rate), `configs` (the GF(2^16) RS(12,4)
configuration and the 4096-stripe mixed batch, measured after the step; see
run_configs) and `cpu_baseline` (the CPU oracle on a bounded sample of the
workload).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1312_5155_gb300.inputs import workload_seed  # noqa: E402

SEED = workload_seed("block_sizes")  # the data and erasures of this RS(10,4) 1 GiB workload

K, M, W = 10, 4, 8
BLOCK = 1 << 20
PACKET = 2048
DATA_BYTES = 1 << 30
REALIZATIONS = ("poly", "vandermonde", "cauchy", "good_cauchy")
PACKET_REALIZATIONS = ("cauchy", "good_cauchy")
METRIC = "encode/decode GB/s (poly vs Cauchy) RS(10,4) on 1 GB300, % HBM peak; serve p50/p99"
WORKLOAD = ("RS(10,4) GF(2^8), 1 GiB data in 102 stripes of 10 x 1 MiB blocks; per realization "
            "(poly, vandermonde, cauchy P=2 KiB, good cauchy P=2 KiB): batched encode of all stripes + batched "
            "decode with 4 seeded erasures per stripe (min-read)")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per stripe of
# each bench kernel, from one ncu capture of `python bench.py --profile-case
# <op> --profile-stripes 300` (one launch over 300 stripes, whose output is
# nine times the L2, so the writes are counted too) divided by 300; a bench
# launch streams 102 stripes, so its traffic is 102 x this.  Valid only for
# the kernel sources with the recorded digest (kernel_digest()); otherwise
# reported as null.
TRAFFIC = {"digest": "8338f3452c2613f7", "per_stripe": {
    "poly_encode": 14589864,
    "poly_decode": 14579256,
    "vandermonde_encode": 14574843,
    "vandermonde_decode": 14573149,
    "cauchy_encode": 14575301,
    "cauchy_decode": 14897019,
    "good_cauchy_encode": 14576605,
    "good_cauchy_decode": 14966968}}


def kernel_digest() -> str:
    """sha256 over the CUDA/C++ sources and the build script of the library."""
    import hashlib

    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1312_5155_gb300")
    csrc = os.path.join(pkg, "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".hpp", ".cuh", ".cu", ".cpp")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    with open(os.path.join(pkg, "build.py"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(op_name: str, stripes: int):
    per = TRAFFIC["per_stripe"].get(op_name)
    if per is None or TRAFFIC["digest"] != kernel_digest():
        return None
    return int(per * stripes)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def n_stripes():
    return DATA_BYTES // (K * BLOCK)


def bench_config() -> dict:
    """The workload's description, the same on both arms of the bench."""
    return {"workload": WORKLOAD, "k": K, "m": M, "w": W, "block_bytes": BLOCK, "packet_bytes": PACKET,
            "stripes_per_gpu": n_stripes(), "realizations": list(REALIZATIONS),
            "l2": "inputs (4 x 1.4 GiB) larger than L2; no flush"}


def global_stripe(rank: int, s: int, per_rank: int) -> int:
    """Stripe s of rank r is stripe r*per_rank + s of the world's data stream:
    ranks shard the stripes with no overlap (weak scaling)."""
    return rank * per_rank + s


def max_over_ranks(value: float, world: int, device) -> float:
    """Slowest rank's time (every rank gets it); no-op for one rank."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(bytes_per_rank: int, world: int, seconds: float) -> float:
    """Units processed by all ranks / the slowest rank's time."""
    return world * bytes_per_rank / seconds


def op_bytes(op: str) -> int:
    return (K + M) * BLOCK  # encode: read k, write m; decode (e = m, min-read): read k, write e


# ---------------------------------------------------------------- our arm
class Workload:
    """Device-resident stripes and the batches that encode / decode them."""

    def __init__(self, rank: int, device, tune: bool = True):
        import torch

        from paper_1312_5155_gb300 import autotune, inputs, rs

        self.S = n_stripes()
        self.n = K + M
        seed = SEED
        self.bufs, self.batches, self.codes, self.ers, self.ops, self.shapes = {}, {}, {}, [], {}, {}
        data = torch.empty((self.S, K, BLOCK), dtype=torch.uint8, device=device)
        for s in range(self.S):
            gs = global_stripe(rank, s, self.S)
            data[s] = inputs.random_bytes_torch(seed, gs * K * BLOCK, K * BLOCK, device).view(K, BLOCK)
        self.ers = [inputs.erasure_pattern(seed, global_stripe(rank, s, self.S), self.n, M) for s in range(self.S)]
        for real in REALIZATIONS:
            code = rs.Code(K, M, W, real, packet_bytes=PACKET if real in PACKET_REALIZATIONS else None)
            # data and parity blocks of all stripes in two contiguous tensors
            dbuf = data.clone()
            pbuf = torch.empty((self.S, M, BLOCK), dtype=torch.uint8, device=device)
            rows = [list(dbuf[s]) + list(pbuf[s]) for s in range(self.S)]
            buf = (dbuf, pbuf)
            enc_ops = [(code, "encode", [], rows[s], BLOCK) for s in range(self.S)]
            dec_ops = [(code, "decode", self.ers[s], rows[s], BLOCK) for s in range(self.S)]
            enc = rs.Batch(self.S)
            enc.set(enc_ops)
            dec = rs.Batch(self.S)
            dec.set(dec_ops)
            self.codes[real], self.bufs[real], self.batches[real] = code, buf, (enc, dec)
            self.ops[real] = (enc_ops, dec_ops)
        del data
        torch.cuda.synchronize()
        for real in REALIZATIONS:  # valid parity before any decode
            self.batches[real][0].launch()
        torch.cuda.synchronize()
        # launch shapes chosen by the autotuner (outside any timed region)
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        for real in REALIZATIONS:
            for i, op in enumerate(("encode", "decode")):
                b = self.batches[real][i]
                if tune:
                    key = autotune.make_key(f"batch{self.S}-{op}", real, K, M, W, BLOCK, sms)
                    shape, _ = autotune.tune_batch(b, self.ops[real][i], key=key)
                else:
                    shape = (8, 16, 1)
                self.shapes[f"{real}_{op}"] = list(shape)
        torch.cuda.synchronize()

    def launches(self):
        return sum(b.kernel_count for pair in self.batches.values() for b in pair)

    def block(self, real, s, b):
        dbuf, pbuf = self.bufs[real]
        return dbuf[s, b] if b < K else pbuf[s, b - K]


def run_ours(args, rank, world, device):
    import torch

    wl = Workload(rank, device, tune=not args.no_tune)
    st = torch.cuda.current_stream()
    names = [(real, op) for real in REALIZATIONS for op in ("encode", "decode")]

    def step(ev=None):
        for i, (real, op) in enumerate(names):
            if ev is not None:
                ev[i].record(st)
            wl.batches[real][0 if op == "encode" else 1].launch()
        if ev is not None:
            ev[len(names)].record(st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    sampler = ClockSampler(device.index if device.index is not None else 0) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # the NVTX range marks the timed region for profilers (ncu --nvtx
    # --nvtx-include "timed_steps/")
    torch.cuda.nvtx.range_push("timed_steps")
    t0.record(st)
    for i in range(args.steps):
        step(evs[i])
    t1.record(st)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop() if sampler else None
    total_ms = t0.elapsed_time(t1)
    op_ms = {nm: sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps for i, nm in enumerate(names)}
    total_ms = max_over_ranks(total_ms, world, device)
    status = {real: (b[0].poll_status(), b[1].poll_status()) for real, b in wl.batches.items()}

    S = wl.S
    step_bytes = sum(S * op_bytes(op) for _, op in names)
    value = whole_job_rate(args.steps * step_bytes, world, total_ms * 1e-3) / 1e9
    user = world * args.steps * len(names) * S * K * BLOCK / (total_ms * 1e-3) / 1e9
    peak, kind = peaks()
    ops = {}
    for (real, op), ms in op_ms.items():
        gbs = S * op_bytes(op) / (ms * 1e-3) / 1e9
        ops[f"{real}_{op}"] = {"gbs": round(gbs, 1), "ms_per_launch": round(ms, 4),
                               "frac_of_hbm": round(gbs / peak, 4), "user_gbs": round(S * K * BLOCK / ms / 1e6, 1)}
    dom = max(op_ms, key=op_ms.get)
    dom_gbs = ops[f"{dom[0]}_{dom[1]}"]["gbs"]
    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": f"synthetic (SplitMix64 uniform-random bytes, seed {SEED:#x})",
        "config": bench_config(),
        "user_gbs": round(user, 2),
        "ops": ops,
        "roofline": {"bound": "hbm", "kernel": f"{dom[0]}_{dom[1]}", "achieved": dom_gbs, "peak": peak,
                     "peak_kind": kind, "unit": "GB/s", "frac": round(dom_gbs / peak, 4),
                     "traffic": traffic_per_launch(f"{dom[0]}_{dom[1]}", S),
                     "algorithmic_bytes": S * op_bytes(dom[1]), "kernel_digest": kernel_digest()},
        "launch_shapes": {k2: {"consumer_warps": v[0], "depth": v[1], "ctas_per_sm": v[2]}
                          for k2, v in wl.shapes.items()},
        "gpu_launches": args.steps * wl.launches(),
        "device_status": status,
        "clocks": clocks,
    }
    return result, wl


def staging_layout(ers, S):
    """Where the end-to-end decode finds each stripe's blocks.  A storage
    server receives the blocks a min-read decode reads (the first K
    survivors by block index) into a staging buffer and returns the rebuilt
    ones from another: stripe s's read blocks are rows s*K .. s*K+K-1 of
    the input staging buffer (in block order), its erased blocks rows
    s*M .. of the output one.  Returns, per stripe, (read blocks, erased
    blocks); needs e = M erasures per stripe (then every block is either
    read or rebuilt)."""
    out = []
    for s in range(S):
        read = [b for b in range(K + M) if b not in ers[s]][:K]
        if len(ers[s]) != M or len(read) != K:
            raise ValueError("the end-to-end step needs M erasures per stripe")
        out.append((read, sorted(ers[s])))
    return out


E2E_CHUNKS = 4  # stripe chunks per request stream: transfers of one overlap the coding of another


def run_e2e(args, wl, device):
    """The same step with host buffers, through the C ABI.  Per realization
    two independent request streams, as a storage server sees them:
      - encode: the data goes host->device, is encoded (batched launches)
        and the parity comes back;
      - decode: the read blocks of the stored stripes (the first K survivors
        of every stripe, received into one staging buffer) go host->device,
        are decoded and the rebuilt blocks come back (staging_layout).
    Copies are transfers between pinned host memory and the device, inside
    the timed region: host -> device as copy-engine transfers, device ->
    host through rs_copy_blocks, on a copy engine or by the library's
    gather kernel: after the warm-up the K timed steps run once with each
    path and the line reports the faster run (both are in `paths_gbs`): how the link shares its two directions differs between GB300
    boxes (engine both ways 128 GB/s in total on one, 343 on another; a
    copy engine one way and the kernel the other 296 and 289; one direction
    alone about 211 GB/s host -> device and 193 device -> host).  Each request stream has its own device and host
    buffers (the decode reads the parity stored by the warm-up's encode) and
    works in E2E_CHUNKS chunks of stripes: chunk c's input copy and launch go
    on one CUDA stream, its output copy on a second one, so the host->device
    copies, the kernels and the device->host copies of different chunks,
    streams and realizations overlap.  The returned blocks are checked after
    the timed region."""
    import torch

    from paper_1312_5155_gb300 import rs

    S = wl.S
    main = torch.cuda.current_stream()
    layout = staging_layout(wl.ers, S)
    bounds = [(S * c // E2E_CHUNKS, S * (c + 1) // E2E_CHUNKS) for c in range(E2E_CHUNKS)]
    bounds = [b for b in bounds if b[1] > b[0]]
    flows, checks = [], []
    for real in REALIZATIONS:
        dbuf, pbuf = wl.bufs[real]
        code = wl.codes[real]
        hd = dbuf.cpu().pin_memory()                                       # data
        hp = torch.empty((S, M, BLOCK), dtype=torch.uint8).pin_memory()   # encode's parity output
        stored = pbuf.cpu()                                                # stored parity
        hin = torch.empty((S, K, BLOCK), dtype=torch.uint8).pin_memory()  # decode input staging
        hout = torch.empty((S, M, BLOCK), dtype=torch.uint8).pin_memory()  # decode output staging
        truth = torch.empty((S, M, BLOCK), dtype=torch.uint8)
        for st_i, (read, er) in enumerate(layout):
            for i, b in enumerate(read):
                hin[st_i, i] = hd[st_i, b] if b < K else stored[st_i, b - K]
            for j, b in enumerate(er):
                truth[st_i, j] = hd[st_i, b] if b < K else stored[st_i, b - K]
        din = torch.empty((S, K, BLOCK), dtype=torch.uint8, device=device)
        dout = torch.empty((S, M, BLOCK), dtype=torch.uint8, device=device)
        for op, hi, di, do, ho in (("encode", hd, dbuf, pbuf, hp), ("decode", hin, din, dout, hout)):
            chunks = []
            for a, b in bounds:
                ops = []
                for st_i in range(a, b):
                    if op == "encode":
                        rows = list(dbuf[st_i]) + list(pbuf[st_i])
                        ops.append((code, "encode", [], rows, BLOCK))
                    else:
                        read, er = layout[st_i]
                        rows = [None] * (K + M)
                        for i, blk in enumerate(read):
                            rows[blk] = din[st_i, i]
                        for j, blk in enumerate(er):
                            rows[blk] = dout[st_i, j]
                        ops.append((code, "decode", wl.ers[st_i], rows, BLOCK))
                batch = rs.Batch(b - a)
                batch.set_launch(*wl.shapes[f"{real}_{op}"])
                batch.set(ops)
                chunks.append(dict(a=a, b=b, batch=batch, done=None))
            flows.append(dict(hi=hi, di=di, do=do, ho=ho, chunks=chunks,
                              sin=torch.cuda.Stream(device=device), sout=torch.cuda.Stream(device=device)))
        checks.append((real, hp, hout, truth))

    def step(d2h_engine):
        h2d = d2h = 0
        for f in flows:
            for ch in f["chunks"]:
                a, b = ch["a"], ch["b"]
                with torch.cuda.stream(f["sin"]):
                    f["di"][a:b].copy_(f["hi"][a:b], non_blocking=True)
                    if ch["done"] is not None:  # the previous step's output copy has read the outputs
                        f["sin"].wait_event(ch["done"])
                    ch["batch"].launch(stream=f["sin"])
                    coded = torch.cuda.Event()
                    coded.record(f["sin"])
                f["sout"].wait_event(coded)
                with torch.cuda.stream(f["sout"]):
                    # device -> host on a copy engine (one range) or by the
                    # gather kernel, whichever the probe below measured faster
                    src, dst = f["do"][a:b], f["ho"][a:b]
                    rs.rs_copy_blocks([dst.data_ptr()], [src.data_ptr()], [src.numel()], stream=f["sout"],
                                      engine_min_bytes=1 if d2h_engine else rs.ENGINE_NEVER)
                    ch["done"] = torch.cuda.Event()
                    ch["done"].record(f["sout"])
                h2d += f["di"][a:b].numel()
                d2h += f["do"][a:b].numel()
        return h2d, d2h

    def join():
        for f in flows:
            for st in (f["sin"], f["sout"]):
                ev = torch.cuda.Event()
                ev.record(st)
                main.wait_event(ev)

    def timed(steps, d2h_engine):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(main)
        for f in flows:
            f["sin"].wait_event(t0)
            f["sout"].wait_event(t0)
        for _ in range(steps):
            sizes = step(d2h_engine)
        join()
        t1.record(main)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), sizes

    # warm-up, then the K steps once with each device -> host path, keeping
    # the faster run: how the host link shares its two directions between
    # copy engines and SM traffic differs between machines (one GB300 machine:
    # engine both ways 128 GB/s in total, engine + gather kernel 296;
    # another: 343 and 289)
    timed(max(1, args.warmup), True)
    runs = {mode: timed(args.steps, mode == "copy_engine") for mode in ("copy_engine", "gather_kernel")}
    path_ms = {mode: r[0] for mode, r in runs.items()}
    d2h_mode = min(path_ms, key=path_ms.get)
    ms, (h2d, d2h) = runs[d2h_mode]
    for real, hp, hout, truth in checks:
        if not torch.equal(hout, truth):
            raise RuntimeError(f"e2e: {real} decode returned wrong blocks")
        if not torch.equal(hp, wl.bufs[real][1].cpu()):
            raise RuntimeError(f"e2e: {real} encode returned wrong parity")
    for f in flows:
        for ch in f["chunks"]:
            ch["batch"].close()
    step_bytes = len(REALIZATIONS) * 2 * S * (K + M) * BLOCK
    return {"value": round(args.steps * step_bytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "d2h_path": d2h_mode,
            "paths_gbs": {k: round(args.steps * step_bytes / (v * 1e-3) / 1e9, 1) for k, v in path_ms.items()}}


SERVE_LOAD = 0.5      # fraction of the measured saturation rate
SERVE_SECONDS = 3.0


def _serial_capacity(pool, codes, seconds: float = 1.0) -> float:
    """Requests/s of the serial per-request path with every request waiting."""
    import torch

    from paper_1312_5155_gb300 import inputs, serve

    reqs = serve.make_requests(inputs.workload_seed("serving") + 7, 1e9, 1.0, max_requests=2000)
    for r in reqs:
        r.arrival = 0.0
    payloads = serve.make_payloads(reqs, pool)
    results = serve.make_results(reqs, pool)
    serve.serial_run(reqs[:20], payloads, results, codes, torch.device("cuda"))
    t0 = time.perf_counter()
    serve.serial_run(reqs, payloads, results, codes, torch.device("cuda"), max_wall=seconds)
    dt = time.perf_counter() - t0
    return sum(1 for r in reqs if r.done >= 0) / dt


def run_configs():
    """The other configurations of the metric, measured in the same run so
    that they come with the bench line: RS(12,4) over GF(2^16) with 4 MiB
    blocks (poly, Cauchy, good Cauchy; batched encode and decode with 1..4
    erasures, 42 stripes), five points of the block-size and k studies
    (RS(10,4) at 4 KiB, 64 KiB and 16 MiB blocks, RS(6,3) and RS(20,4) at
    1 MiB; poly, Vandermonde, good Cauchy) and the 4096-stripe mixed batch
    (codes (6,3) (10,4) (12,4) (20,4), blocks of 4 KiB - 8 MiB, 30 %
    decodes; batched, replayed from a CUDA graph, and as a loop of
    per-stripe calls, with per-op completion latency).  GB/s of algorithmic bytes; frac = of the
    HBM peak."""
    import torch

    from paper_1312_5155_gb300 import sweep
    peak, kind = peaks()
    out = {"hbm_peak_gbs": peak, "peak_kind": kind}
    gf16 = {}
    for r in sweep.gf16_blocks(emit=False):
        row = {}
        for key, v in r.items():
            if isinstance(v, dict) and "gbs" in v:
                row[key] = {"gbs": v["gbs"], "frac": round(v["gbs"] / peak, 3)}
        gf16[r["realization"]] = row
    out["gf16_rs12_4_4MiB_42stripes"] = gf16
    torch.cuda.empty_cache()
    # points of the block-size and k studies: 1 GiB of data each, m seeded
    # erasures per decode, tuned launch shapes
    seed = workload_seed("block_sizes")
    pts = {}
    for (k, m, B) in ((10, 4, 4 << 10), (10, 4, 64 << 10), (10, 4, 16 << 20), (6, 3, 1 << 20), (20, 4, 1 << 20)):
        stripes = max(1, (1 << 30) // (k * B))
        row = {}
        for real in ("poly", "vandermonde", "good_cauchy"):
            r = sweep._batch_pair(real, 8, k, m, B, stripes, seed, m, tag="bench-")
            row[real] = {op: {"gbs": r[op]["gbs"], "frac": round(r[op]["gbs"] / peak, 3)} for op in ("encode", "decode")}
        pts[f"rs{k}_{m}_B{B >> 10}KiB"] = row
        torch.cuda.empty_cache()
    out["block_and_k_points"] = pts
    mb = sweep.mixed_batch(emit=False)
    torch.cuda.empty_cache()
    mb["frac_batched"] = round(mb["batched"]["gbs"] / peak, 3)
    mb["frac_graph_replay"] = round(mb["graph_replay"]["gbs"] / peak, 3)
    out["mixed_batch_4096"] = mb
    return out


def run_serve():
    """The metric's serving part on this GPU (configuration 5's request mix):
    the continuous-batching server (paper_1312_5155_gb300.serve) under Poisson
    arrivals for SERVE_SECONDS at SERVE_LOAD of its saturation rate (the
    highest rate it keeps up with, found by bisection), request latency
    p50 / p99 and served GB/s; then the batched server and the serial
    per-request path at the same offered rate, half of what the serial path
    sustains, and at twice that capacity (the serial path falls behind:
    fewer requests completed within the run, lower GB/s)."""
    from paper_1312_5155_gb300 import inputs, rs, serve

    budget = 32 << 30
    pool = serve.HostPool(2 << 30)
    sat = serve.saturation_rate(budget, pool)
    rate = SERVE_LOAD * sat
    reqs = serve.make_requests(inputs.workload_seed("serving"), rate, SERVE_SECONDS)
    payloads = serve.make_payloads(reqs, pool)
    results = serve.make_results(reqs, pool)
    srv = serve.Server(budget)
    srv.run(reqs, payloads, results)
    summary = serve.summarize(reqs, wall=SERVE_SECONDS)
    codes = {c: rs.Code(c[0], c[1], 8, "poly") for c in serve.CODES}
    cap = _serial_capacity(pool, codes)
    srate = 0.5 * cap
    reqs_b = serve.make_requests(inputs.workload_seed("serving"), srate, SERVE_SECONDS)
    pay_b = serve.make_payloads(reqs_b, pool)
    res_b = serve.make_results(reqs_b, pool)
    srv.run(reqs_b, pay_b, res_b)
    reqs_s = serve.make_requests(inputs.workload_seed("serving"), srate, SERVE_SECONDS)
    serve.serial_run(reqs_s, pay_b, res_b, codes, __import__("torch").device("cuda"),
                     max_wall=SERVE_SECONDS + 5.0)
    # past the serial path's capacity (and below the batched saturation):
    # the batched server keeps up, the serial path falls behind
    orate = min(2.0 * cap, 0.8 * sat)
    over_s = 2.0
    reqs_ob = serve.make_requests(inputs.workload_seed("serving") + 11, orate, over_s)
    pay_o = serve.make_payloads(reqs_ob, pool)
    res_o = serve.make_results(reqs_ob, pool)
    srv.run(reqs_ob, pay_o, res_o)
    reqs_os = serve.make_requests(inputs.workload_seed("serving") + 11, orate, over_s)
    serve.serial_run(reqs_os, pay_o, res_o, codes, __import__("torch").device("cuda"), max_wall=over_s)
    del srv

    def rnd(d):
        return {k: round(v, 4) if isinstance(v, float) else v for k, v in d.items()}

    return {"load": SERVE_LOAD, "rate_req_per_s": round(rate, 1), "saturation_req_per_s": round(sat, 1),
            "seconds": SERVE_SECONDS, "requests": len(reqs), **rnd(summary),
            "vs_serial": {"rate_req_per_s": round(srate, 1), "serial_capacity_req_per_s": round(cap, 1),
                          "requests": len(reqs_b), "batched": rnd(serve.summarize(reqs_b, wall=SERVE_SECONDS)),
                          "serial": rnd(serve.summarize(reqs_s, wall=SERVE_SECONDS))},
            "overload": {"rate_req_per_s": round(orate, 1), "seconds": over_s, "requests": len(reqs_ob),
                         "batched": rnd(serve.summarize(reqs_ob, wall=over_s)),
                         "serial": rnd(serve.summarize(reqs_os, wall=over_s))}}


# ------------------------------------------------------------ oracle arm
def cpu_info() -> dict:
    """Model and clock of the host CPU (lscpu, else /proc/cpuinfo)."""
    info = {"cpu_model": None, "cpu_max_mhz": None, "logical_cpus": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            key, val = key.strip(), val.strip()
            if key == "Model name" and not info["cpu_model"]:
                info["cpu_model"] = val
            elif key == "CPU max MHz":
                info["cpu_max_mhz"] = float(val)
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    if not info["cpu_model"]:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        info["cpu_model"] = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    if info["cpu_max_mhz"] is None:
        try:
            with open("/sys/devices/system/cpu/cpu0/cpufreq/cpuinfo_max_freq") as f:
                info["cpu_max_mhz"] = int(f.read()) / 1000.0
        except (OSError, ValueError):
            pass
    return info


def _oracle_stripe_pass(s: int) -> float:
    """The oracle (as it stands) on one whole stripe of the workload: each
    realization's encode, then its 4-erasure decode.  Returns seconds."""
    import numpy as np

    from oracle import oracle as O
    from paper_1312_5155_gb300 import inputs

    n = K + M
    b0 = np.zeros((n, BLOCK), dtype=np.uint8)
    b0[:K] = inputs.stripe_blocks(SEED, s, K, BLOCK)
    er = inputs.erasure_pattern(SEED, s, n, M)
    t = time.perf_counter()
    for real in REALIZATIONS:
        b = b0.copy()
        O.encode(real, W, K, M, b, packet_bytes=PACKET)
        b[er] = 0
        O.decode(real, W, K, M, er, b, packet_bytes=PACKET)
    return time.perf_counter() - t


def oracle_run(threads: int, passes_per_thread: int, first: int = 1) -> tuple[float, int]:
    """GB/s of `threads` host threads each running `passes_per_thread`
    stripe passes (stripe indices taken modulo the workload's stripes)."""
    import concurrent.futures as cf

    from oracle import oracle as O

    O.lib()
    nstripes = threads * passes_per_thread
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(_oracle_stripe_pass, [s % n_stripes() for s in range(first, first + nstripes)]))
    dt = time.perf_counter() - t0
    step_bytes = nstripes * len(REALIZATIONS) * 2 * (K + M) * BLOCK
    return step_bytes / dt / 1e9, nstripes


def oracle_sample(seconds_target: float = 12.0, runs: int = 3):
    """The CPU oracle timed as the paper times its codecs (§5.1: the mean of
    3 runs) on whole stripes of the same workload, once with one thread per
    host core and once single-threaded, each run sized to about
    seconds_target / (2 * runs) of wall time."""
    import statistics as stats

    from oracle import oracle as O

    O.lib()
    cores = os.cpu_count() or 1
    t_one = _oracle_stripe_pass(0)
    per_run = seconds_target / (2 * runs)
    all_passes = max(1, int(per_run / max(t_one, 1e-3)))
    one_passes = max(1, int(per_run / max(t_one, 1e-3)))
    multi = [oracle_run(cores, all_passes, first=1 + r * cores * all_passes) for r in range(runs)]
    single = [oracle_run(1, one_passes, first=1 + r * one_passes) for r in range(runs)]
    info = cpu_info()
    return {"value": round(stats.mean(v for v, _ in multi), 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "runs": runs, "per_run_gbs": [round(v, 4) for v, _ in multi],
            "single_thread_gbs": round(stats.mean(v for v, _ in single), 4),
            "single_thread_per_run_gbs": [round(v, 4) for v, _ in single],
            **info,
            "sample": f"whole stripes of the 102 RS(10,4) 1 MiB-block stripes, encode + 4-erasure decode in each "
                      f"of the {len(REALIZATIONS)} realizations per stripe pass; all-core: {runs} runs of {cores} threads x "
                      f"{all_passes} passes (one stripe per thread at a time); single-thread: {runs} runs of "
                      f"{one_passes} passes; value = mean of the all-core runs"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    t_one = _oracle_stripe_pass(0)
    passes = max(1, int(3.0 / max(t_one, 1e-3)))  # about 3 s per step
    for _ in range(args.warmup):
        oracle_run(cores, 1)
    samples = [oracle_run(cores, passes, first=1 + i * cores * passes)[0] for i in range(args.steps)]
    v = statistics.mean(samples)
    base = {"cores": cores, "sample": f"{args.steps} steps of {cores} threads x {passes} whole-stripe passes "
                                      f"(encode + 4-erasure decode in each of the {len(REALIZATIONS)} realizations); value = mean "
                                      f"over the steps", **cpu_info()}
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": f"synthetic (SplitMix64, seed {SEED:#x})",
        "config": bench_config(),
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": base["cores"], "kind": "oracle",
                         "sample": base["sample"], "cpu_model": base["cpu_model"],
                         "cpu_max_mhz": base["cpu_max_mhz"]},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def profile_case(name: str, stripes: int = 16, launches: int = 3, shape=None):
    """One bench kernel for ncu: `stripes` stripes of the bench geometry
    (RS(10,4), 1 MiB blocks; 16 stripes = 224 MiB, larger than L2; 102 =
    the bench's launch), one realization, `launches` batched launches of one
    op (after one encode that makes the parity valid), with the launch
    shape the bench's autotuner chose (or `shape`)."""
    import torch

    from paper_1312_5155_gb300 import autotune, inputs, rs

    real, op = name.rsplit("_", 1)
    seed = SEED
    n = K + M
    # the launch shape the bench's autotuner chose for this op (if cached)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    hit = autotune._load().get(autotune.make_key(f"batch{n_stripes()}-{op}", real, K, M, W, BLOCK, sms))
    if shape is None:
        shape = tuple(hit["shape"]) if hit else (8, 16, 1)
    code = rs.Code(K, M, W, real, packet_bytes=PACKET if real in PACKET_REALIZATIONS else None)
    buf = torch.empty((stripes, n, BLOCK), dtype=torch.uint8, device="cuda")
    buf[:, :K] = inputs.random_bytes_torch(seed, 0, stripes * K * BLOCK, "cuda").view(stripes, K, BLOCK)
    rows = [list(buf[s]) for s in range(stripes)]
    enc = rs.Batch(stripes)
    enc.set_launch(*shape)
    enc.set([(code, "encode", [], rows[s], BLOCK) for s in range(stripes)])
    enc.launch()
    b = enc
    if op == "decode":
        b = rs.Batch(stripes)
        b.set_launch(*shape)
        b.set([(code, "decode", inputs.erasure_pattern(seed, s, n, M), rows[s], BLOCK) for s in range(stripes)])
    for _ in range(launches):
        b.launch()
    torch.cuda.synchronize()
    if b.poll_status() != 0:
        raise SystemExit("device status word set")
    print(f"profile case {name}: {launches} launches of {stripes} stripes, launch shape {shape}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-latency measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the GF(2^16) and 4096-stripe mixed-batch configurations")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--profile-case", default=None,
                    help="run one small kernel case for ncu, e.g. poly_encode, cauchy_decode")
    ap.add_argument("--profile-stripes", type=int, default=16, help="stripes of the --profile-case launch")
    ap.add_argument("--profile-shape", default=None, help="launch shape warps,depth,ctas_per_sm for --profile-case")
    args = ap.parse_args()
    if args.profile_case:
        shape = tuple(int(x) for x in args.profile_shape.split(",")) if args.profile_shape else None
        profile_case(args.profile_case, stripes=args.profile_stripes, shape=shape)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return

    import torch
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)
    result, wl = run_ours(args, rank, world, device)
    if not args.no_e2e:
        e2e = run_e2e(args, wl, device)
        if world > 1:
            t = torch.tensor([e2e["value"]], device=device)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MIN)
            e2e["value"] = round(float(t.item()) * world, 2)
        result["e2e"] = e2e
    if rank == 0 and not args.no_serve:
        result["serve"] = run_serve()
    if rank == 0 and world == 1 and not args.no_configs:
        del wl
        torch.cuda.empty_cache()
        result["configs"] = run_configs()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = oracle_sample()
        else:
            result["cpu_baseline"] = None
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
