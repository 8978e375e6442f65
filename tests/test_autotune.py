"""Autotuner selection and cache logic, with a fake batch (no GPU)."""
import json

from paper_1312_5155_gb300 import autotune


class FakeBatch:
    def __init__(self, cost):
        self.cost = cost
        self.shape = None
        self.sets = 0

    def set_launch(self, *shape):
        self.shape = shape

    def set(self, ops):
        self.sets += 1

    def launch(self):
        pass


def test_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("RS_GB300_TUNE_CACHE", str(tmp_path / "tune.json"))
    cost = {(16, 8, 1): 3.0, (8, 8, 2): 1.5, (4, 16, 2): 2.0}
    # the two best shapes are tried again with one and two column groups;
    # forcing one group is slower, forcing two no faster than the default
    forced = {(8, 8, 2, 1): 2.5, (8, 8, 2, 2): 1.5, (4, 16, 2, 1): 2.4, (4, 16, 2, 2): 2.0}
    b = FakeBatch(cost)
    monkeypatch.setattr(autotune, "time_launch", lambda launch, reps=5: {**cost, **forced}[b.shape])
    key = autotune.make_key("encode", "poly", 10, 4, 8, 1 << 20, 152)
    best, res = autotune.tune_batch(b, [], key=key, candidates=list(cost))
    assert best == (8, 8, 2) and b.shape == (8, 8, 2)
    assert set(res) == set(cost) | set(forced)
    d = json.loads((tmp_path / "tune.json").read_text())
    assert d[key]["shape"] == [8, 8, 2]
    # second call: cache hit, no timing
    monkeypatch.setattr(autotune, "time_launch", lambda *a, **k: (_ for _ in ()).throw(AssertionError))
    b2 = FakeBatch(cost)
    best2, _ = autotune.tune_batch(b2, [], key=key, candidates=list(cost))
    assert best2 == (8, 8, 2) and b2.shape == (8, 8, 2) and b2.sets == 1


def test_key_buckets_block_sizes():
    k1 = autotune.make_key("decode", "cauchy", 10, 4, 8, 1 << 20, 152)
    k2 = autotune.make_key("decode", "cauchy", 10, 4, 8, (1 << 20) + 4096, 152)
    k3 = autotune.make_key("decode", "cauchy", 10, 4, 8, 1 << 21, 152)
    assert k1 == k2 != k3


def test_column_groups_can_win(tmp_path, monkeypatch):
    """A forced column-group count that beats the default is kept, with the
    group count as the shape's fourth element."""
    monkeypatch.setenv("RS_GB300_TUNE_CACHE", str(tmp_path / "tune.json"))
    cost = {(16, 8, 1): 3.0, (8, 8, 2): 1.5, (4, 16, 2): 2.0,
            (8, 8, 2, 1): 1.7, (8, 8, 2, 2): 1.2, (4, 16, 2, 1): 2.2, (4, 16, 2, 2): 2.1}
    b = FakeBatch(cost)
    monkeypatch.setattr(autotune, "time_launch", lambda launch, reps=5: cost[b.shape])
    key = autotune.make_key("decode", "poly", 10, 4, 8, 64 << 10, 152)
    best, _ = autotune.tune_batch(b, [], key=key, candidates=[(16, 8, 1), (8, 8, 2), (4, 16, 2)])
    assert best == (8, 8, 2, 2) and b.shape == (8, 8, 2, 2)
    d = json.loads((tmp_path / "tune.json").read_text())
    assert d[key]["shape"] == [8, 8, 2, 2]
