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


class StepSim:
    """Stands in for Simulator in tune_on_steps: a launch shape and per-shape step times; one shape has no
    co-resident launch (its steps raise, as the library does)."""

    def __init__(self, cost, infeasible=()):
        self.shape = (4, 2)
        self.cost = cost
        self.infeasible = set(infeasible)
        self.ran = []

    def tuning(self, rowg=0, blocks_per_sm=0, autotune_next_step=False):
        if rowg:
            self.shape = (rowg, self.shape[1])
        if blocks_per_sm:
            self.shape = (self.shape[0], blocks_per_sm)
        return self.shape, [0.0] * 8

    def run(self, j):
        from paper_2609_25653_b300.ipcsim import IpcError
        if self.shape in self.infeasible:
            raise IpcError(-3, "PCG kernel cannot be made resident")
        self.ran.append((self.shape, j))
        return self.cost(self.shape, j)


def test_tune_on_steps_keeps_the_smallest_total_over_all_steps():
    # (2, 1) wins the first step but loses the sum; (8, 1) cannot launch
    def cost(shape, j):
        base = {(1, 1): 9, (2, 1): 5, (4, 1): 7, (8, 1): 1, (1, 2): 8, (2, 2): 7, (4, 2): 6, (8, 2): 9}[shape]
        return base + (0 if shape == (2, 1) and j == 0 else (4 if shape == (2, 1) else 0))
    sim = StepSim(cost, infeasible={(8, 1)})
    shape, ms = autotune.tune_on_steps(sim, sim.run, 3)
    assert shape == (4, 2) and sim.shape == (4, 2)
    assert ms[4 * 0 + 3] == -1.0                      # (8, 1) skipped
    assert ms[4 * 0 + 1] == 5 + 9 + 9                 # (2, 1): every step counted
    assert ms[4 * 1 + 2] == 18                        # (4, 2)
    assert {s for s, _ in sim.ran} == {(r, b) for r in (1, 2, 4, 8) for b in (1, 2)} - {(8, 1)}
    assert all(len([1 for s, _ in sim.ran if s == sh]) == 3 for sh in {s for s, _ in sim.ran})


def test_cached_applies_a_stored_shape_only(tmp_path):
    cache = str(tmp_path / "tune.json")
    sim = FakeSim(5000)
    assert autotune.cached(sim, 0, cache_path=cache) is False and sim.calls == []
    autotune.record(FakeSim(5000, chosen=(8, 1)), 0, cache_path=cache, ms=[1.0] * 8)
    assert json.load(open(cache)).popitem()[1]["ms"] == [1.0] * 8
    hit = FakeSim(5000)
    assert autotune.cached(hit, 0, cache_path=cache) is True and hit.calls == [(8, 1, False)]
