"""GPU parity at the benchmark's full size: the RS(10,4) workload of 1 GiB of
data in 102 stripes of 10 x 1 MiB blocks, in all four realizations, run
through the same batches, launch shapes (autotuned) and erasure patterns that
bench.py times.

The oracle cannot redo 4 x 1.4 GiB in test time, so it checks samples:
every stripe on 64 random byte columns (in the symbol layout each byte
offset is a codeword of its own) or on one random super-packet (in the
Cauchy packet layouts the super-packets are independent), and three whole
stripes per realization.  The check runs after the decode, on all 14
blocks: the rebuilt blocks must equal the original data and parity, and
the blocks left alone must hold the batched encode's parity."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_5155_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rows(wl, real, s, sel):
    """All n blocks of stripe s at the byte index `sel` (a CUDA index
    tensor or a slice), on the host."""
    import torch
    dbuf, pbuf = wl.bufs[real]
    both = torch.cat([dbuf[s][:, sel], pbuf[s][:, sel]], dim=0)
    return both.cpu().numpy()


def test_bench_workload_sampled_parity():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_1312_5155_gb300 import build
    build.build()
    K, M, W, B, P = bench.K, bench.M, bench.W, bench.BLOCK, bench.PACKET
    seed = bench.SEED
    wl = bench.Workload(0, torch.device("cuda:0"), tune=True)
    rng = np.random.default_rng(0x5A11)
    whole = {0, wl.S // 2, wl.S - 1}
    for real in bench.REALIZATIONS:
        enc, dec = wl.batches[real]
        enc.launch()
        torch.cuda.synchronize()
        assert enc.poll_status() == 0
        for s in range(wl.S):
            for b in wl.ers[s]:
                wl.block(real, s, b).fill_(0xE1)
        dec.launch()
        torch.cuda.synchronize()
        assert dec.poll_status() == 0
    for s in range(wl.S):
        data = inputs.random_bytes(seed, bench.global_stripe(0, s, wl.S) * K * B, K * B).reshape(K, B)
        for real in bench.REALIZATIONS:
            if real in bench.PACKET_REALIZATIONS:
                sp = int(rng.integers(0, B // (W * P)))
                sel = slice(sp * W * P, (sp + 1) * W * P)
                ref = np.zeros((K + M, W * P), dtype=np.uint8)
                ref[:K] = data[:, sel]
            else:
                cols = np.sort(rng.choice(B, 64, replace=False))
                sel = torch.from_numpy(cols).cuda()
                ref = np.zeros((K + M, 64), dtype=np.uint8)
                ref[:K] = data[:, cols]
            O.encode(real, W, K, M, ref, packet_bytes=P)
            got = _rows(wl, real, s, sel)
            assert np.array_equal(got, ref), (real, s, wl.ers[s])
            if s in whole:
                ref = np.zeros((K + M, B), dtype=np.uint8)
                ref[:K] = data
                O.encode(real, W, K, M, ref, packet_bytes=P)
                assert np.array_equal(_rows(wl, real, s, slice(0, B)), ref), (real, s, "whole stripe")
