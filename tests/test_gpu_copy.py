"""GPU: rs_copy_blocks moves many byte ranges between page-locked host memory
and device memory (small ranges by the gather kernel, one launch per 512 of
them; large ones on the copy engines), bit-exact."""
import numpy as np
import pytest

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


def _ranges(n, seed, maxlen):
    u = inputs.uniform01(inputs.shape_draws(seed, 0, n))
    return [int(x * maxlen) for x in u]


@pytest.mark.parametrize("engine", ["default", "all", "none"])
@pytest.mark.parametrize("direction", ["h2d", "d2h", "d2d"])
def test_copy_ranges_bit_exact(rs, direction, engine):
    import torch
    n = 700  # small ranges: two kernel launches
    lens = _ranges(n, 3, 70000)
    lens[5] = 0
    lens[6] = 1
    lens[7] = 15
    slot = 80 * 1024
    # three copy-engine sized ranges interleaved with the small ones
    big = [(4 << 20) + 16, 5 << 20, (4 << 20) + 4096 + 3]
    big_slot = 6 << 20
    total = n * slot + len(big) * big_slot
    src_np = inputs.random_bytes(9, 0, total)
    host = torch.from_numpy(src_np.copy()).pin_memory()
    dev = torch.empty(total, dtype=torch.uint8, device="cuda")
    if direction == "h2d":
        src, dst = host, dev
        dst.fill_(0xEE)
    elif direction == "d2h":
        dev.copy_(host)
        src, dst = dev, torch.full((total,), 0xEE, dtype=torch.uint8).pin_memory()
    else:
        dev.copy_(host)
        src, dst = dev, torch.full((total,), 0xEE, dtype=torch.uint8, device="cuda")
    # small range i: slot i of src -> slot (n - 1 - i) of dst; big range j:
    # big slot j -> big slot (len(big) - 1 - j)
    plan = [(i * slot, (n - 1 - i) * slot, ln) for i, ln in enumerate(lens)]
    nb = len(big)
    for j, ln in enumerate(big):
        plan.insert(200 * j + 1, (n * slot + j * big_slot, n * slot + (nb - 1 - j) * big_slot, ln))
    engine_min = {"default": 0, "all": 1, "none": rs.ENGINE_NEVER}[engine]
    rs.rs_copy_blocks([dst.data_ptr() + d for _, d, _ in plan], [src.data_ptr() + a for a, _, _ in plan],
                      [ln for _, _, ln in plan], engine_min_bytes=engine_min)
    torch.cuda.synchronize()
    got = dst.cpu().numpy()
    want = np.full(total, 0xEE, dtype=np.uint8)
    for a, d, ln in plan:
        want[d:d + ln] = src_np[a:a + ln]
    assert np.array_equal(got, want)


def test_copy_rejects_pageable_and_misaligned(rs):
    import torch
    dev = torch.empty(4096, dtype=torch.uint8, device="cuda")
    pageable = torch.empty(4096, dtype=torch.uint8)
    with pytest.raises(rs.RSError) as ei:
        rs.rs_copy_blocks([dev.data_ptr()], [pageable.data_ptr()], [4096])
    assert ei.value.status == 1 and "page-locked" in str(ei.value)
    pinned = torch.empty(4096, dtype=torch.uint8).pin_memory()
    with pytest.raises(rs.RSError) as ei:
        rs.rs_copy_blocks([dev.data_ptr() + 8], [pinned.data_ptr()], [64])
    assert "aligned" in str(ei.value)
    with pytest.raises(rs.RSError):
        rs.rs_copy_blocks([dev.data_ptr()], [dev.data_ptr() + 16], [64])  # overlaps itself
    rs.rs_copy_blocks([], [], [])  # nothing to do
