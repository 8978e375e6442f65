"""Seeded synthetic inputs: uniform-random block bytes and erasure patterns.

This module holds no Reed-Solomon arithmetic.  It is the one module that both
the CPU oracle's callers (tests, bench) and the GPU path's callers use, so that
every comparison runs on identical bytes.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a counter-based generator: word i
(0-based) of the stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15),
where mix is the SplitMix64 finaliser.  Because every word depends only on its
index, any slice of a multi-gigabyte stream can be produced directly, which is
what the full-size sampled parity checks rely on.

Byte streams are the little-endian bytes of consecutive words: byte o of a
stream is byte (o % 8) of word (o // 8).

The paper measures on random in-memory data (§5.1); the named workloads below
mirror its RS(10,4) GF(2^8) setting and the block sizes of §5.2.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Stream tags: distinct sub-streams derived from one workload seed.
TAG_DATA = 0x0
TAG_ERASURE = 0xA5A5A5A5A5A5A5A5
TAG_SHAPE = 0x5A5A5A5A5A5A5A5A


# The synthetic workloads and the index of their seed: one RS(10,4) stripe
# of 64 KiB blocks; RS(6,3) / RS(10,4) over 1 GiB at block sizes 4 KiB -
# 64 MiB; RS(12,4) over GF(2^16) with 4 MiB blocks; 4096 stripes of mixed
# codes and sizes in one batch; Poisson requests to the serving loop.
WORKLOADS = {"single_stripe": 1, "block_sizes": 2, "gf16_blocks": 3, "mixed_batch": 4, "serving": 5}


def stream_seed(index: int) -> int:
    """Seed of stream ``index``: 0x5EED0000 + index."""
    return 0x5EED0000 + int(index)


def workload_seed(name: str) -> int:
    """Seed of a named workload (see WORKLOADS)."""
    return stream_seed(WORKLOADS[name])


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def splitmix64_words(seed: int, start: int, count: int) -> np.ndarray:
    """Words ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = idx * np.uint64(GAMMA) + np.uint64(seed & MASK64)
        return _mix_np(x)


def splitmix64_scalar(seed: int, index: int) -> int:
    """Word ``index`` of stream ``seed`` in plain Python integers."""
    z = (seed + (index + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def random_bytes(seed: int, offset: int, nbytes: int) -> np.ndarray:
    """Bytes ``offset .. offset+nbytes-1`` of the byte stream of ``seed``."""
    if nbytes <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = offset // 8
    w1 = (offset + nbytes + 7) // 8
    words = splitmix64_words(seed, w0, w1 - w0).astype("<u8", copy=False)
    b = words.view(np.uint8)
    s = offset - 8 * w0
    return b[s:s + nbytes].copy()


def stripe_blocks(seed: int, stripe: int, k: int, block_bytes: int,
                  col0: int = 0, ncols: int | None = None) -> np.ndarray:
    """Data blocks of one stripe as a (k, ncols) uint8 array.

    The data of a workload is one long byte stream cut into stripes of k blocks
    of ``block_bytes``: block j of stripe s starts at byte (s*k + j)*block_bytes.
    ``col0``/``ncols`` select a column window of every block (for sampling).
    """
    if ncols is None:
        ncols = block_bytes - col0
    out = np.empty((k, ncols), dtype=np.uint8)
    for j in range(k):
        out[j] = random_bytes(seed ^ TAG_DATA, (stripe * k + j) * block_bytes + col0, ncols)
    return out


def erasure_pattern(seed: int, stripe: int, n: int, e: int) -> list[int]:
    """First ``e`` entries of a Fisher-Yates shuffle of 0..n-1 (Durstenfeld).

    Draw i of stripe s is word s*n + i of the erasure sub-stream; step i
    (from n-1 down to 1) swaps entry i with entry draw_i mod (i+1).
    """
    if not 0 <= e <= n:
        raise ValueError("need 0 <= e <= n")
    words = splitmix64_words(seed ^ TAG_ERASURE, stripe * n, n)
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = int(words[i]) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:e]


def shape_draws(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform 64-bit draws for workload shapes (codes, sizes, ops)."""
    return splitmix64_words(seed ^ TAG_SHAPE, start, count)


def uniform01(words: np.ndarray) -> np.ndarray:
    """Map 64-bit draws to floats in [0, 1) using their top 53 bits."""
    return (words >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


MIXED_CODES = ((6, 3), (10, 4), (12, 4), (20, 4))


def mixed_batch_shapes(seed: int, stripes: int = 4096, min_bytes: int = 4096, max_bytes: int = 8 << 20,
                       decode_share: float = 0.30):
    """Stripe shapes of the mixed batch: per stripe (k, m, B, e, offset).

    (k, m) uniform over MIXED_CODES; B log-uniform on [min_bytes, max_bytes],
    rounded down to a multiple of 4 KiB (at least 4 KiB); a decode with
    probability decode_share, its erasure count e uniform in 1..m (e = 0:
    an encode).  Stripe s draws words 4s .. 4s+3 of the shape sub-stream.
    The stripes lie one after another in one buffer, each as k data blocks
    then m parity blocks; `offset` is the stripe's first byte in it, and data
    block j of stripe s holds the bytes offset + j*B .. of the data stream
    (random_bytes(seed, offset + j*B, B)).
    """
    import math

    u = uniform01(shape_draws(seed, 0, 4 * stripes)).reshape(stripes, 4)
    out, off = [], 0
    lo, hi = math.log(min_bytes), math.log(max_bytes)
    for s in range(stripes):
        k, m = MIXED_CODES[int(u[s, 0] * len(MIXED_CODES)) % len(MIXED_CODES)]
        B = int(math.exp(lo + u[s, 1] * (hi - lo))) // 4096 * 4096
        B = max(4096, B)
        e = 1 + int(u[s, 3] * m) % m if u[s, 2] < decode_share else 0
        out.append((k, m, B, e, off))
        off += (k + m) * B
    return out


# ---------------------------------------------------------------- torch form
def random_bytes_torch(seed: int, offset: int, nbytes: int, device="cpu"):
    """Same bytes as :func:`random_bytes`, generated with torch int64 ops.

    Used to fill large device buffers without a host round trip.  int64
    multiplication wraps modulo 2^64, and logical right shifts are an
    arithmetic shift followed by a mask, so the words equal the uint64 ones.
    """
    import torch

    if nbytes <= 0:
        return torch.zeros(0, dtype=torch.uint8, device=device)

    def s64(v):
        v &= MASK64
        return v - (1 << 64) if v >= (1 << 63) else v

    def lsr(x, s):
        return (x >> s) & ((1 << (64 - s)) - 1)

    w0 = offset // 8
    w1 = (offset + nbytes + 7) // 8
    x = torch.arange(w0 + 1, w1 + 1, dtype=torch.int64, device=device)
    x = x * s64(GAMMA) + s64(seed)
    x = (x ^ lsr(x, 30)) * s64(MIX1)
    x = (x ^ lsr(x, 27)) * s64(MIX2)
    x = x ^ lsr(x, 31)
    b = x.view(torch.uint8)
    s = offset - 8 * w0
    return b[s:s + nbytes]
