"""Continuous-batching request server for RS encode/decode on one GPU.

Requests (encode or decode of one stripe of some code and block size)
arrive over time.  The loop:
  - admits arrived requests while their stripe fits the device-memory
    budget (a first-fit arena of pre-allocated device memory: buffers stay
    resident and are reused, nothing is allocated per request);
  - as soon as one of `streams` launch slots is free, packs every admitted
    request into one batch (rs_batch_set + rs_batch_launch: one persistent
    launch per kernel group) on that slot's stream, preceded by the
    host->device transfer of the requests' input blocks and followed by the
    device->host transfer of their output blocks (rs_copy_blocks: one launch
    per direction for the whole batch);
  - polls the slots' completion events; a finished request frees its arena
    memory, which admits the next arrivals.
Requests arriving while earlier batches run are admitted and launched on
another stream, so their transfers and kernels overlap on the device
(continuous batching, not a queue drained one batch at a time).

Latency of a request = host time of completion (its batch's event observed)
- its arrival time.  The serial baseline runs every request alone
(rs_encode / rs_decode, copies, synchronise) in arrival order.
"""
from __future__ import annotations

import argparse
import bisect
import json
import math
import os
import sys
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs

CODES = [(6, 3), (10, 4), (12, 4), (20, 4)]
ALIGN = 256


# ----------------------------------------------------------------- arena
class Arena:
    """First-fit allocator over [0, capacity) with coalescing free list."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.free = [(0, capacity)]  # sorted (offset, size)
        self.used = 0

    def alloc(self, size: int):
        size = (size + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, sz) in enumerate(self.free):
            if sz >= size:
                if sz == size:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + size, sz - size)
                self.used += size
                return off, size
        return None

    def release(self, off: int, size: int):
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, size))
        self.used -= size
        # coalesce with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)


# --------------------------------------------------------------- requests
@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    k: int
    m: int
    op: str                 # "encode" / "decode"
    block_bytes: int
    erasures: list = field(default_factory=list)
    payload: int = 0        # index of the host payload stripe
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    off: int = -1
    size: int = 0


def make_requests(seed: int, rate: float, seconds: float, median: int = 256 << 10, sigma: float = 1.0,
                  cap: int = 64 << 20, decode_frac: float = 0.25, max_requests: int | None = None):
    """Poisson arrivals at `rate`/s for `seconds`; block sizes lognormal
    (median, sigma) rounded down to 4 KiB, capped; codes uniform over CODES;
    `decode_frac` decodes with e uniform in 1..m."""
    n_max = max_requests or int(rate * seconds * 1.5 + 100)
    u = inputs.uniform01(inputs.shape_draws(seed, 0, 6 * n_max)).reshape(n_max, 6)
    t = 0.0
    out = []
    for i in range(n_max):
        t += -math.log(1.0 - u[i, 0]) / rate
        if t > seconds:
            break
        k, m = CODES[int(u[i, 1] * len(CODES)) % len(CODES)]
        # Box-Muller from two uniforms for the lognormal size
        z = math.sqrt(-2.0 * math.log(1.0 - u[i, 2])) * math.cos(2.0 * math.pi * u[i, 3])
        B = int(median * math.exp(sigma * z))
        B = max(4096, min(cap, B // 4096 * 4096))
        op = "decode" if u[i, 4] < decode_frac else "encode"
        er = []
        if op == "decode":
            e = 1 + int(u[i, 5] * m) % m
            er = inputs.erasure_pattern(seed, i, k + m, e)
        out.append(Request(rid=i, arrival=t, k=k, m=m, op=op, block_bytes=B, erasures=er))
    return out


def io_blocks(req: Request):
    """(blocks copied host->device, blocks copied device->host)."""
    n = req.k + req.m
    if req.op == "encode":
        return list(range(req.k)), list(range(req.k, n))
    read = [b for b in range(n) if b not in req.erasures][:req.k]
    return read, list(req.erasures)


def algorithmic_bytes(req: Request) -> int:
    if req.op == "encode":
        return (req.k + req.m) * req.block_bytes
    return (req.k + len(req.erasures)) * req.block_bytes


# ----------------------------------------------------------------- server
class Server:
    def __init__(self, budget_bytes: int, streams: int = 4, max_batch: int = 256, device=None):
        import torch

        from . import rs

        self.torch, self.rs = torch, rs
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.budget = budget_bytes
        self.arena = Arena(budget_bytes)
        self.mem = torch.empty(budget_bytes, dtype=torch.uint8, device=self.device)
        self.base = self.mem.data_ptr()
        self.codes = {}
        for (k, m) in CODES:
            self.codes[(k, m)] = rs.Code(k, m, 8, "poly")
        self.max_batch = max_batch
        self.slots = []
        for _ in range(streams):
            self.slots.append({"stream": torch.cuda.Stream(device=self.device),
                               "batch": rs.Batch(max_batch), "event": torch.cuda.Event(),
                               "reqs": None})

    def _block_view(self, off: int, b: int, B: int):
        start = off + b * ((B + 15) // 16 * 16)
        return self.mem[start:start + B]

    def run(self, requests, payloads, results=None, time_limit: float | None = None):
        """Serve `requests` (sorted by arrival) in real time.  payloads[i] is a
        pinned uint8 host tensor (n, B) holding the stripe of request i (for
        decodes: the codeword with erased blocks ignored); results[i], when
        given, receives the output blocks (pinned host tensor (n_out, B))."""
        torch = self.torch
        pending = list(requests)
        admitted = []
        pi = 0
        t0 = time.perf_counter()
        done = 0
        while done < len(requests):
            now = time.perf_counter() - t0
            if time_limit and now > time_limit:
                break
            # 1. admit arrivals that fit the budget (in arrival order)
            while pi < len(pending) and pending[pi].arrival <= now:
                r = pending[pi]
                n = r.k + r.m
                need = n * ((r.block_bytes + 15) // 16 * 16)
                if need > self.budget:
                    raise ValueError(f"request {r.rid} needs more than the whole budget")
                got = self.arena.alloc(need)
                if got is None:
                    break
                r.off, r.size = got
                r.admitted = now
                admitted.append(r)
                pi += 1
            # 2. launch admitted requests on a free slot
            if admitted:
                for slot in self.slots:
                    if slot["reqs"] is None:
                        batch_reqs = admitted[:self.max_batch]
                        admitted = admitted[self.max_batch:]
                        self._launch(slot, batch_reqs, payloads, results)
                        break
            # 3. retire finished slots
            for slot in self.slots:
                if slot["reqs"] is not None and slot["event"].query():
                    tdone = time.perf_counter() - t0
                    for r in slot["reqs"]:
                        r.done = tdone
                        self.arena.release(r.off, r.size)
                        done += 1
                    slot["reqs"] = None
            if not admitted and (pi >= len(pending) or pending[pi].arrival > time.perf_counter() - t0):
                busy = any(s["reqs"] is not None for s in self.slots)
                if not busy and pi < len(pending):
                    # idle until the next arrival
                    wait = pending[pi].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.001))
        # a run cut short by time_limit: let the batches in flight finish and
        # give back the memory of everything admitted (those requests count
        # as complete only if their batch had finished)
        for slot in self.slots:
            if slot["reqs"] is not None:
                slot["event"].synchronize()
                tdone = time.perf_counter() - t0
                for r in slot["reqs"]:
                    r.done = tdone
                    self.arena.release(r.off, r.size)
                slot["reqs"] = None
        for r in admitted:
            self.arena.release(r.off, r.size)
        return requests

    def _launch(self, slot, reqs, payloads, results):
        """One batch on the slot's stream: the input blocks of every request
        in (encode: the k data rows; decode: the k rows a min-read decode
        reads), one launch per kernel group, the output blocks out (parity
        rows; rebuilt rows).  Both transfers are one rs_copy_blocks call each,
        all ranges on the gather kernel (one launch reading / writing the
        page-locked host buffers: no per-range set-up cost), with the ranges
        of consecutive rows of a request merged.  Block pointers are
        computed from the arena base, so no tensor views are made per block."""
        torch, rs = self.torch, self.rs
        st = slot["stream"]
        ops = []
        src, dst, nb = [], [], []
        for r in reqs:
            n, B = r.k + r.m, r.block_bytes
            Bp = (B + 15) // 16 * 16
            base = self.base + r.off
            hp = payloads[r.rid].data_ptr()
            for i, b in enumerate(io_blocks(r)[0]):
                _add_range(dst, src, nb, base + b * Bp, hp + b * B, B, join=i > 0)
            ops.append((self.codes[(r.k, r.m)], r.op, r.erasures, [base + b * Bp for b in range(n)], B))
        with torch.cuda.stream(st):
            rs.rs_copy_blocks(dst, src, nb, stream=st, engine_min_bytes=rs.ENGINE_NEVER)
            slot["batch"].set(ops, stream=st)
            slot["batch"].launch(stream=st)
            if results is not None:
                src, dst, nb = [], [], []
                for r in reqs:
                    B = r.block_bytes
                    Bp = (B + 15) // 16 * 16
                    base = self.base + r.off
                    res = results[r.rid].data_ptr()
                    for j, b in enumerate(io_blocks(r)[1]):
                        _add_range(dst, src, nb, res + j * B, base + b * Bp, B, join=j > 0)
                rs.rs_copy_blocks(dst, src, nb, stream=st, engine_min_bytes=rs.ENGINE_NEVER)
            slot["event"].record(st)
        slot["reqs"] = reqs


def _add_range(dst, src, nb, d, s, n, join=True):
    """Append a copy range, extending the previous one when `join` (the two
    belong to the same host buffer) and both ends follow on from it.  Ranges
    of different host buffers stay apart even when adjacent in memory: a
    copy-engine transfer must not cross from one allocation into another."""
    if join and nb and dst[-1] + nb[-1] == d and src[-1] + nb[-1] == s:
        nb[-1] += n
    else:
        dst.append(d)
        src.append(s)
        nb.append(n)


def serial_run(requests, payloads, results, codes, device, max_wall: float | None = None):
    """Every request alone, in arrival order (copies, one launch, sync).
    One device buffer per codeword length, sized for the largest block of
    the run.  With max_wall, requests not started by then stay incomplete
    (an overloaded serial path falls behind without bound)."""
    import torch
    t0 = time.perf_counter()
    cap = max((r.block_bytes for r in requests), default=16)
    cap = (cap + 15) // 16 * 16
    bufs = {}
    for r in requests:
        now = time.perf_counter() - t0
        if max_wall is not None and now > max_wall:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        n, B = r.k + r.m, r.block_bytes
        if n not in bufs:
            bufs[n] = torch.empty((n, cap), dtype=torch.uint8, device=device)
        buf = bufs[n]
        blocks = [buf[b, :B] for b in range(n)]
        h2d, d2h = io_blocks(r)
        for b in h2d:
            blocks[b].copy_(payloads[r.rid][b], non_blocking=True)
        code = codes[(r.k, r.m)]
        if r.op == "encode":
            code.encode(blocks[:r.k], blocks[r.k:], B)
        else:
            code.decode(r.erasures, blocks, B)
        for j, b in enumerate(d2h):
            results[r.rid][j].copy_(blocks[b], non_blocking=True)
        torch.cuda.synchronize()
        r.done = time.perf_counter() - t0
    return requests


def summarize(requests, wall: float | None = None):
    lat = np.array([r.done - r.arrival for r in requests if r.done >= 0])
    done = [r for r in requests if r.done >= 0]
    if not len(lat):
        return {"completed": 0}
    span = wall or (max(r.done for r in done) - min(r.arrival for r in done))
    return {"completed": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "gbs": sum(algorithmic_bytes(r) for r in done) / span / 1e9, "span_s": span}


class HostPool:
    """One pinned host buffer of seeded random bytes; every request's payload
    (and result) is a view into it.  Content is irrelevant to timing; the
    correctness tests build their own per-request payloads."""

    def __init__(self, nbytes: int, seed: int = 0x5EED0005):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        chunk = min(nbytes, 64 << 20)
        pattern = torch.from_numpy(inputs.random_bytes(seed, 0, chunk))
        for off in range(0, nbytes, chunk):
            n = min(chunk, nbytes - off)
            self.buf[off:off + n].copy_(pattern[:n])
        self.nbytes = nbytes

    def view(self, rid: int, rows: int, cols: int):
        need = rows * cols
        if need > self.nbytes:
            raise ValueError("pool smaller than one request")
        off = (rid * 7919 * 4096) % (self.nbytes - need + 1) // 16 * 16
        return self.buf[off:off + need].view(rows, cols)


def make_payloads(requests, pool: "HostPool"):
    return {r.rid: pool.view(r.rid, r.k + r.m, r.block_bytes) for r in requests}


def make_results(requests, pool: "HostPool | None" = None):
    import torch
    if pool is None:
        return {r.rid: torch.empty((len(io_blocks(r)[1]), r.block_bytes), dtype=torch.uint8).pin_memory()
                for r in requests}
    return {r.rid: pool.view(r.rid + 1, len(io_blocks(r)[1]), r.block_bytes) for r in requests}


def drain_rate(budget: int, pool: "HostPool", seconds: float = 2.0, seed: int = 0x5EED0005, srv=None) -> float:
    """Requests/s the batched server completes when every request is already
    waiting (all arrivals at t = 0): an upper bound, since waiting requests
    fill the largest batches."""
    reqs = make_requests(seed, 1e9, 1.0, max_requests=int(400 * seconds))
    for r in reqs:
        r.arrival = 0.0
    payloads = make_payloads(reqs, pool)
    srv = srv or Server(budget)
    srv.run(reqs[:50], payloads)  # warm-up
    t0 = time.perf_counter()
    srv.run(reqs, payloads)
    dt = time.perf_counter() - t0
    return len(reqs) / dt


def keeps_up(srv, pool, rate: float, seconds: float, p50_light_ms: float, seed: int = 0x5EED0006,
             factor: float = 10.0):
    """One Poisson run at `rate`: the server keeps up when every request
    completes within 50 ms of the end of the arrivals and the p99 latency
    stays within `factor` times the p50 latency at light load."""
    reqs = make_requests(seed, rate, seconds)
    payloads = make_payloads(reqs, pool)
    srv.run(reqs, payloads)
    s = summarize(reqs)
    last = max((r.done for r in reqs), default=0.0)
    ok = s.get("completed", 0) == len(reqs) and last <= seconds + 0.05 and s["p99_ms"] <= factor * p50_light_ms
    return ok, s


def saturation_rate(budget: int, pool: "HostPool", probe_seconds: float = 1.0, probes: int = 6,
                    seed: int = 0x5EED0005) -> float:
    """The highest Poisson arrival rate (requests/s) the batched server keeps
    up with (keeps_up), found by bisection between 5 % and 100 % of the
    drain rate.  Loads at or below it are sustained: p99 within a small
    multiple (10x) of the light-load p50."""
    srv = Server(budget)
    top = drain_rate(budget, pool, seed=seed, srv=srv)
    light = make_requests(seed + 1, 0.05 * top, probe_seconds)
    srv.run(light, make_payloads(light, pool))
    p50_light = summarize(light)["p50_ms"]
    lo, hi = 0.05, 1.0
    for _ in range(probes):
        mid = 0.5 * (lo + hi)
        ok, _ = keeps_up(srv, pool, mid * top, probe_seconds, p50_light)
        if ok:
            lo = mid
        else:
            hi = mid
    del srv
    return lo * top


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--budget-gib", type=float, default=32.0)
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--rates", default="0.1,0.3,0.5,0.7,0.9,1.0,1.2", help="fractions of the saturation rate")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--serial", action="store_true", help="also run the serial per-request path")
    a = ap.parse_args()
    budget = int(a.budget_gib * (1 << 30))
    pool = HostPool(2 << 30)
    sat = saturation_rate(budget, pool)
    out = {"saturation_req_per_s": sat, "seconds": a.seconds, "runs": []}
    srv = Server(budget, streams=a.streams)
    codes = None
    for frac in [float(x) for x in a.rates.split(",")]:
        rate = frac * sat
        reqs = make_requests(inputs.workload_seed("serving"), rate, a.seconds)
        payloads = make_payloads(reqs, pool)
        results = make_results(reqs, pool)
        srv.run(reqs, payloads, results, time_limit=a.seconds + 30.0)
        row = {"rate_frac": frac, "rate": rate, "offered": len(reqs), "batched": summarize(reqs, wall=a.seconds)}
        if a.serial:
            import torch
            from . import rs
            codes = codes or {c: rs.Code(c[0], c[1], 8, "poly") for c in CODES}
            reqs2 = make_requests(inputs.workload_seed("serving"), rate, a.seconds)
            serial_run(reqs2, payloads, results, codes, torch.device("cuda"), max_wall=a.seconds + 10.0)
            row["serial"] = summarize(reqs2, wall=a.seconds)
        out["runs"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
