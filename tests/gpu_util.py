"""Helpers for the GPU tests: device blocks with 16-byte aligned rows."""
import numpy as np


def device_blocks(host: np.ndarray):
    """Copy an (n, B) uint8 array to the GPU as n row views whose starts are
    16-byte aligned (rows padded to a multiple of 16 bytes)."""
    import torch
    n, B = host.shape
    Bp = max(16, (B + 15) // 16 * 16)
    buf = torch.zeros((n, Bp), dtype=torch.uint8, device="cuda")
    if B:
        buf[:, :B] = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    rows = [buf[i, :B] for i in range(n)]
    return buf, rows


def to_host(buf, B: int) -> np.ndarray:
    return buf[:, :B].cpu().numpy()
