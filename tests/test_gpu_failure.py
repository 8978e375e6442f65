"""Failure detection on the GPU without a fault: a bounded device-side wait
is made to run out (CTA 0's producer withholds its copies through a test
hook), the kernel records RS_ETIMEOUT in the status word and returns, and
the context stays usable for correct work afterwards."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests.gpu_util import device_blocks, to_host

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs
    build.build()
    k, m, w, B = 10, 4, 8, 1 << 20
    host = np.zeros((k + m, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(inputs.stream_seed(1), 9, k, B)
    ref = host.copy()
    O.poly_encode(w, k, m, ref)
    code = rs.Code(k, m, w, "poly")
    rs.rs_set_wait_limit(code.handle, 2_000_000)  # 2 ms
    buf, rows = device_blocks(host)
    rs.rs_inject_fault(code.handle, 1)
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    status = code.poll_status()
    assert status == 0x101  # consumer wait on a slot that was never filled
    # the hook applies to one launch only and the context is intact
    rs.rs_set_wait_limit(code.handle, 0)
    code.encode(rows[:k], rows[k:], B)
    torch.cuda.synchronize()
    assert code.poll_status() == 0
    assert np.array_equal(to_host(buf, B), ref)
