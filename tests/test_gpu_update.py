"""GPU: rs_update (§3.2's update remark: the parity diff is the encode of the
data diff) for every realization, bit-exact against the oracle's encode of
the updated data."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs
from tests.gpu_util import device_blocks, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_5155_gb300 import build, rs as rsmod
    build.build()
    return rsmod


# (realization, w, k, m, B, packet)
CASES = [("poly", 8, 10, 4, (1 << 20) + 48, None), ("poly", 8, 6, 3, 5000, None), ("poly", 16, 12, 4, 40002, None),
         ("poly", 8, 20, 8, 70000, None), ("vandermonde", 8, 10, 4, 65536 + 16, None),
         ("cauchy", 8, 10, 4, 8 * 2048 * 4, 2048), ("cauchy", 16, 6, 3, 16 * 512 * 2, 512),
         ("good_cauchy", 8, 10, 4, 8 * 2048 * 4, 2048),
         ("poly_matrix", 8, 7, 5, 30000, None), ("poly_bitmatrix", 8, 10, 4, 8 * 1024 * 3, 1024)]


@pytest.mark.parametrize("real,w,k,m,B,pkt", CASES)
def test_update_equals_encode_of_new_data(rs, real, w, k, m, B, pkt):
    import torch
    code = rs.Code(k, m, w, real, packet_bytes=pkt)
    host = np.zeros((k + m, B), dtype=np.uint8)
    host[:k] = inputs.stripe_blocks(inputs.stream_seed(4), 3, k, B)
    O.encode(real, w, k, m, host, packet_bytes=pkt or 2048)
    buf, rows = device_blocks(host)
    for step, index in enumerate([0, k - 1, k // 2]):
        new = inputs.stripe_blocks(inputs.stream_seed(4), 100 + step, 1, B)[0]
        delta = np.bitwise_xor(host[index], new)
        host[index] = new
        O.encode(real, w, k, m, host, packet_bytes=pkt or 2048)  # expected parity of the new data
        dbuf, drows = device_blocks(delta[None, :])
        code.update(index, drows[0], rows[k:], B)
        torch.cuda.synchronize()
        assert code.poll_status() == 0
        assert np.array_equal(to_host(buf, B)[k:], host[k:]), (index, step)


def test_update_argument_errors(rs):
    import torch
    code = rs.Code(10, 4, 8, "poly")
    t = torch.zeros((6, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.RSError):
        code.update(10, t[0], list(t[1:5]), 4096)       # index out of range
    with pytest.raises(rs.RSError):
        code.update(0, t[1], list(t[1:5]), 4096)        # delta overlaps a parity block
    code.update(3, t[0], list(t[1:5]), 0)               # nothing to do
