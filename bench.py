#!/usr/bin/env python
"""Encode/decode throughput of the GB300 Reed-Solomon library.

Workload (one step): the RS(10,4) GF(2^8) part of the 1 GiB workload of
§5.2-style experiments: 1 GiB of uniform-random data cut into stripes of 10
blocks x 1 MiB (102 stripes).  For every realization timed, a step encodes
all stripes, then decodes all stripes with m = 4 seeded erasures each
(min-read: k survivors).  Inputs are resident in HBM (1.4 GiB, larger than
L2) when the timed region starts.

value = algorithmic bytes / time, where a stripe encode moves (k+m)*B bytes
and a min-read decode (k+e)*B bytes; `user_gbs` = data bytes k*B per
stripe-op / time.  N > 1 (torchrun): every rank runs the same per-GPU
workload on its own stripes (weak scaling, no collective on the data path);
value = bytes of all ranks / max rank time.

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

K, M, W = 10, 4, 8
BLOCK = 1 << 20
DATA_BYTES = 1 << 30
CONFIG = 2
METRIC = "encode/decode GB/s (poly vs Cauchy) RS(10,4) on 1 GB300, % HBM peak; serve p50/p99"


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(rank: int = 0):
    n = K + M
    stripes = DATA_BYTES // (K * BLOCK)
    return n, stripes


def erasures_for(stripe: int, n: int):
    from paper_1312_5155_gb300 import inputs
    return inputs.erasure_pattern(inputs.config_seed(CONFIG), stripe, n, M)


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, device):
    import torch

    from paper_1312_5155_gb300 import inputs, rs

    n, S = workload(rank)
    seed = inputs.config_seed(CONFIG)
    # rank r processes stripes of its own 1 GiB slice of a world-sized stream
    buf = torch.empty((S, n, BLOCK), dtype=torch.uint8, device=device)
    for s in range(S):
        gs = rank * S + s
        buf[s, :K] = inputs.random_bytes_torch(seed, gs * K * BLOCK, K * BLOCK, device).view(K, BLOCK)
    code = rs.Code(K, M, W, "poly")
    rows = [list(buf[s]) for s in range(S)]
    ers = [erasures_for(rank * S + s, n) for s in range(S)]

    def encode_all():
        for s in range(S):
            code.encode(rows[s][:K], rows[s][K:], BLOCK)

    def decode_all():
        for s in range(S):
            code.decode(ers[s], rows[s], BLOCK)

    # first encode makes the parity valid, so every decode reproduces bytes
    encode_all()
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        encode_all()
        decode_all()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(device.index if device.index is not None else 0) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for i in range(args.steps):
        ev[i][0].record(st)
        encode_all()
        ev[i][1].record(st)
        decode_all()
        ev[i][2].record(st)
    t1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_ms = t0.elapsed_time(t1)
    enc_ms = sum(e[0].elapsed_time(e[1]) for e in ev)
    dec_ms = sum(e[1].elapsed_time(e[2]) for e in ev)
    if world > 1:
        t = torch.tensor([total_ms], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    status = code.poll_status()

    enc_bytes = S * (K + M) * BLOCK
    dec_bytes = S * (K + M) * BLOCK  # k read + e=m written
    step_bytes = enc_bytes + dec_bytes
    value = world * args.steps * step_bytes / (total_ms * 1e-3) / 1e9
    user = world * args.steps * 2 * S * K * BLOCK / (total_ms * 1e-3) / 1e9
    peak, kind = peaks()
    enc_launch_ms = enc_ms / (args.steps * S)
    dec_launch_ms = dec_ms / (args.steps * S)
    enc_gbs = (K + M) * BLOCK / (enc_launch_ms * 1e-3) / 1e9
    dec_gbs = (K + M) * BLOCK / (dec_launch_ms * 1e-3) / 1e9
    dominant = ("poly_decode", dec_gbs, dec_launch_ms) if dec_ms >= enc_ms else ("poly_encode", enc_gbs, enc_launch_ms)
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
        "data": "synthetic (SplitMix64 uniform-random bytes, seed 0x5EED0002)",
        "config": {"workload": "RS(10,4) GF(2^8) poly, 1 GiB data in 102 stripes of 10 x 1 MiB blocks; "
                               "encode + decode (4 seeded erasures, min-read) per stripe",
                   "k": K, "m": M, "w": W, "block_bytes": BLOCK, "stripes_per_gpu": S,
                   "realizations": ["poly"], "l2": "inputs (1.4 GiB) larger than L2; no flush"},
        "user_gbs": round(user, 2),
        "ops": {"poly_encode": {"gbs": round(enc_gbs, 1), "ms_per_launch": round(enc_launch_ms, 5)},
                "poly_decode": {"gbs": round(dec_gbs, 1), "ms_per_launch": round(dec_launch_ms, 5)}},
        "roofline": {"bound": "hbm", "kernel": dominant[0], "achieved": round(dominant[1], 1),
                     "peak": peak, "peak_kind": kind, "unit": "GB/s",
                     "frac": round(dominant[1] / peak, 4), "traffic": None},
        "gpu_launches": args.steps * 2 * S,
        "device_status": status,
        "clocks": clocks,
    }
    return result, (buf, code, rows, ers, S, n)


def run_e2e(args, state, device):
    """Same step with host buffers: H2D inputs, kernels, D2H outputs."""
    import torch

    buf, code, rows, ers, S, n = state
    host = torch.empty((S, n, BLOCK), dtype=torch.uint8).pin_memory()
    host.copy_(buf.cpu())
    st = torch.cuda.current_stream()

    def step():
        h2d = d2h = 0
        buf[:, :K].copy_(host[:, :K], non_blocking=True)
        h2d += S * K * BLOCK
        for s in range(S):
            code.encode(rows[s][:K], rows[s][K:], BLOCK)
        host[:, K:].copy_(buf[:, K:], non_blocking=True)
        d2h += S * M * BLOCK
        for s in range(S):
            er = ers[s]
            surv = [b for b in range(n) if b not in er][:K]
            for b in surv:
                buf[s, b].copy_(host[s, b], non_blocking=True)
            h2d += K * BLOCK
            code.decode(er, rows[s], BLOCK)
            for b in er:
                host[s, b].copy_(buf[s, b], non_blocking=True)
            d2h += M * BLOCK
        return h2d, d2h

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(args.steps):
        h2d, d2h = step()
    t1.record(st)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    step_bytes = 2 * S * (K + M) * BLOCK
    return {"value": round(args.steps * step_bytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


# ------------------------------------------------------------ oracle arm
def oracle_sample(seconds_target: float = 12.0):
    """Time the CPU oracle (as it stands) on whole stripes of the same
    workload, one stripe per host thread, until about seconds_target."""
    import concurrent.futures as cf

    import numpy as np

    from oracle import oracle as O
    from paper_1312_5155_gb300 import inputs

    O.lib()
    n = K + M
    seed = inputs.config_seed(CONFIG)
    cores = os.cpu_count() or 1

    def one(s):
        b = np.zeros((n, BLOCK), dtype=np.uint8)
        b[:K] = inputs.stripe_blocks(seed, s, K, BLOCK)
        t = time.perf_counter()
        O.poly_encode(W, K, M, b)
        er = inputs.erasure_pattern(seed, s, n, M)
        b[er] = 0
        O.poly_decode(W, K, M, er, b)
        return time.perf_counter() - t

    # measure one stripe, then size the parallel sample
    t_one = one(0)
    per_thread = max(1, int(seconds_target / max(t_one, 1e-3) / 2))
    nstripes = min(cores * per_thread, 102)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        list(ex.map(one, range(1, 1 + nstripes)))
    dt = time.perf_counter() - t0
    step_bytes = nstripes * 2 * (K + M) * BLOCK
    return {"value": round(step_bytes / dt / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{nstripes} of the 102 RS(10,4) 1 MiB-block stripes, poly encode + 4-erasure decode, "
                      f"one stripe per thread on {cores} host threads ({dt:.1f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    samples = []
    for _ in range(args.warmup):
        oracle_sample(3.0)
    for _ in range(args.steps):
        samples.append(oracle_sample(6.0))
    v = statistics.mean(s["value"] for s in samples)
    base = samples[-1]
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (SplitMix64, seed 0x5EED0002)",
        "config": {"workload": "RS(10,4) GF(2^8) poly, 1 GiB data in 102 stripes of 10 x 1 MiB blocks; "
                               "encode + decode (4 seeded erasures) per stripe", "k": K, "m": M, "w": W,
                   "block_bytes": BLOCK},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": base["cores"], "kind": "oracle",
                         "sample": base["sample"]},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

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
    result, state = run_ours(args, rank, world, device)
    e2e = run_e2e(args, state, device)
    if world > 1:
        t = torch.tensor([e2e["value"]], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MIN)
        e2e["value"] = round(float(t.item()) * world, 2)
    result["e2e"] = e2e
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
