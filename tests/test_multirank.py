"""The N > 1 bench path on CPU with the gloo backend (world size 2): ranks
shard stripes without overlap, the timing is the max over ranks, and the
whole-job value counts every rank's bytes."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1312_5155_gb300 import inputs
    S = 3
    stripes = [bench.global_stripe(rank, s, S) for s in range(S)]
    first = inputs.stripe_blocks(inputs.stream_seed(2), stripes[0], 2, 16)[0].tolist()
    t = bench.max_over_ranks(10.0 + rank, world, torch.device("cpu"))
    out[rank] = (stripes, first, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    s0, f0, t0 = res[0]
    s1, f1, t1 = res[1]
    assert set(s0).isdisjoint(s1) and sorted(s0 + s1) == list(range(6))
    assert f0 != f1  # different data on different ranks
    assert t0 == t1 == 11.0  # both ranks see the slowest rank's time
    import bench
    assert bench.whole_job_rate(100, 2, 2.0) == 100.0
