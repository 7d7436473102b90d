"""Host logic of the PCG launch-shape autotuner (paper_2609_25653_b300/autotune.py), no GPU: a cache miss
asks the next step to time every shape, record() stores the choice per (GPU, precision, size bucket), and a
later prepare() applies it."""
import json

from paper_2609_25653_b300 import autotune


class FakeSim:
    """Stands in for Simulator: records the sim_tuning calls the autotuner makes."""

    def __init__(self, n_nodes, chosen=(2, 1)):
        self.n_nodes = n_nodes
        self.calls = []
        self.chosen = chosen

    def tuning(self, rowg=0, blocks_per_sm=0, autotune_next_step=False):
        self.calls.append((rowg, blocks_per_sm, autotune_next_step))
        return self.chosen, [0.5, 0.4, 0.3, 0.6, 0.7, 0.8, 0.9, 1.0]


def test_miss_then_record_then_hit(tmp_path):
    cache = str(tmp_path / "tune.json")
    sim = FakeSim(10336, chosen=(2, 1))
    assert autotune.prepare(sim, 1, cache_path=cache) is False
    assert sim.calls == [(0, 0, True)]  # the next step times every shape
    got = autotune.record(sim, 1, cache_path=cache)
    assert got == {"rowg": 2, "blocks_per_sm": 1}
    data = json.load(open(cache))
    assert len(data) == 1
    (key, entry), = data.items()
    assert "mixed" in key and "nodes<=16384" in key
    assert entry["rowg"] == 2 and entry["blocks_per_sm"] == 1 and len(entry["ms"]) == 8
    again = FakeSim(12000)  # same size bucket, same precision: cache hit
    assert autotune.prepare(again, 1, cache_path=cache) is True
    assert again.calls == [(2, 1, False)]


def test_keys_separate_precision_and_size(tmp_path):
    cache = str(tmp_path / "tune.json")
    autotune.prepare(FakeSim(10336), 1, cache_path=cache)
    autotune.record(FakeSim(10336, chosen=(4, 2)), 1, cache_path=cache)
    fp64 = FakeSim(10336)
    assert autotune.prepare(fp64, 0, cache_path=cache) is False  # other precision: miss
    big = FakeSim(131488)
    assert autotune.prepare(big, 1, cache_path=cache) is False  # other size bucket: miss
    autotune.record(FakeSim(131488, chosen=(8, 2)), 1, cache_path=cache)
    assert len(json.load(open(cache))) == 2
    hit = FakeSim(131488)
    assert autotune.prepare(hit, 1, cache_path=cache) is True and hit.calls == [(8, 2, False)]


def test_unreadable_cache_is_a_miss(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    sim = FakeSim(100)
    assert autotune.prepare(sim, 0, cache_path=str(cache)) is False
    autotune.record(sim, 0, cache_path=str(cache))  # rewritten whole
    assert len(json.load(open(cache))) == 1
