"""Launch-shape autotuner for the stripe kernels.

A launch shape is (consumer warps per CTA, ring depth, CTAs per SM[,
columns per thread]):
  - consumer warps set the tile width: a tile covers consumer_warps x 32
    threads x 32 columns of every block (1 KiB per warp at w = 8,
    2 KiB at w = 16), and every thread owns 32 columns (64 in the
    two-group kernels); the kernel caps the count at what its registers
    allow;
  - ring depth is how many block slices are in flight per CTA (the unroll
    depth of the shared-memory pipeline);
  - CTAs per SM sets the persistent grid (SMs x CTAs per SM);
  - columns per thread: one or two groups of 32 (the kernels' G); absent =
    the library's choice by block size.
The tuner times every candidate shape on the device (CUDA events, after
warm-up) for one batch and keeps the fastest.  Results are cached in a JSON
file keyed by (op, realization, k, m, w, block-size bucket, SM count).
"""
from __future__ import annotations

import json
import math
import os
import threading

CANDIDATES = [(16, 8, 1), (16, 12, 1), (15, 5, 1), (15, 4, 1), (15, 3, 1), (12, 6, 1), (12, 4, 1), (12, 3, 1),
              (8, 16, 1), (8, 8, 2), (8, 12, 2), (4, 16, 2), (4, 8, 3), (4, 8, 4), (2, 8, 4)]
_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build",
                              "autotune.json")
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("RS_GB300_TUNE_CACHE", _DEFAULT_CACHE)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def make_key(op: str, realization: str, k: int, m: int, w: int, block_bytes: int, sms: int) -> str:
    bucket = int(math.log2(max(block_bytes, 1)))
    return f"{op}/{realization}/k{k}/m{m}/w{w}/B2^{bucket}/sm{sms}"


def time_launch(launch, reps: int = 5, warmup: int = 2) -> float:
    """Mean milliseconds of `launch()` on the current stream."""
    import torch
    for _ in range(warmup):
        launch()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        launch()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(batch, ops, key: str | None = None, candidates=None, reps: int = 5, use_cache: bool = True,
               group_search: bool = True):
    """Pick the fastest launch shape for `batch` running `ops` (the list
    given to Batch.set): every candidate (warps, depth, CTAs per SM) with
    the columns per thread chosen by block size, then the two best with one
    and with two 32-column groups forced (a fourth element of the shape).
    Leaves the batch set with the winning shape and returns (shape,
    {shape: ms})."""
    candidates = list(candidates or CANDIDATES)
    if key and use_cache:
        with _lock:
            hit = _load().get(key)
        if hit:
            shape = tuple(hit["shape"])
            batch.set_launch(*shape)
            batch.set(ops)
            return shape, {shape: hit["ms"]}
    results = {}
    for shape in candidates:
        batch.set_launch(*shape)
        batch.set(ops)
        results[shape] = time_launch(batch.launch, reps=reps)
    # columns per thread: the two best shapes again with one and with two
    # 32-column groups per thread forced (the default picks by block size)
    if group_search:
        for shape in sorted(results, key=results.get)[:2]:
            if len(shape) > 3:
                continue
            for g in (1, 2):
                s4 = tuple(shape) + (g,)
                batch.set_launch(*s4)
                batch.set(ops)
                results[s4] = time_launch(batch.launch, reps=reps)
    best = min(results, key=results.get)
    batch.set_launch(*best)
    batch.set(ops)
    if key:
        with _lock:
            d = _load()
            d[key] = {"shape": list(best), "ms": results[best],
                      "all": {",".join(map(str, s)): v for s, v in results.items()}}
            _store(d)
    return best, results
