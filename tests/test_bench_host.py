"""Host-side logic of bench.py: the staging layout of the end-to-end
decode (which blocks a min-read decode reads and rebuilds)."""
import pytest

import bench
from paper_1312_5155_gb300 import inputs


def test_staging_layout_reads_the_first_k_survivors():
    K, M = bench.K, bench.M
    S = 40
    ers = [inputs.erasure_pattern(inputs.stream_seed(2), s, K + M, M) for s in range(S)]
    lay = bench.staging_layout(ers, S)
    assert len(lay) == S
    for s, (read, er) in enumerate(lay):
        assert read == sorted(set(range(K + M)) - set(ers[s]))[:K]
        assert er == sorted(ers[s])
        # every block is read or rebuilt, once
        assert sorted(read + er) == list(range(K + M))


def test_staging_layout_needs_m_erasures():
    with pytest.raises(ValueError):
        bench.staging_layout([[0]], 1)
