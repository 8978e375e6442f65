"""Host-side logic of bench.py: the runs of blocks a min-read decode reads,
copied host->device in the end-to-end measurement."""
import bench
from paper_1312_5155_gb300 import inputs


def expand(runs):
    return [i for a, b in runs for i in range(a, b)]


def test_read_runs_cover_the_first_k_survivors():
    K, M = bench.K, bench.M
    S = 40
    ers = [inputs.erasure_pattern(inputs.config_seed(2), s, K + M, 1 + s % M) for s in range(S)]
    data, par = bench.read_runs(ers, S)
    want_d, want_p = [], []
    for s in range(S):
        read = sorted(set(range(K + M)) - set(ers[s]))[:K]
        want_d += [s * K + b for b in read if b < K]
        want_p += [s * M + b - K for b in read if b >= K]
    assert expand(data) == want_d
    assert expand(par) == want_p
    # runs are maximal: no two touch
    for runs in (data, par):
        for (a0, b0), (a1, b1) in zip(runs, runs[1:]):
            assert b0 < a1


def test_read_runs_without_erasures_is_one_data_run():
    data, par = bench.read_runs([[] for _ in range(5)], 5)
    assert data == [(0, 5 * bench.K)]
    assert par == []
