"""Host logic of the batched step's autotuner, on the CPU: a fake batch
(whose step time depends on the candidate applied to it) stands in for
``sim_batch_*``, and the device synchronisation is a no-op."""
import json
import time

import pytest

from paper_1412_4933_gb300 import autotune, pedsim as P, workloads as WL

torch = pytest.importorskip("torch")


class FakeBatch:
    """Records the calls the tuner makes; stepping sleeps 20 µs per step
    times the candidate's cost."""
    made = 0

    def __init__(self, scenarios, stream=None, cost=None):
        FakeBatch.made += 1
        self.cost = cost
        self.variant = None
        self.tiling = None
        self.calls = []
        self.closed = False

    def set_variant(self, v):
        self.variant = v
        self.tiling = None
        self.calls.append(("variant", v))

    def set_tiling(self, tw, th, cps):
        self.tiling = (tw, th, cps)
        self.calls.append(("tiling", tw, th, cps))

    def step(self, n):
        key = (self.variant,) + (self.tiling or (0, 0, 0))
        time.sleep(2e-5 * n * self.cost[key])

    def close(self):
        self.closed = True


@pytest.fixture
def fake_env(monkeypatch, tmp_path):
    made = []

    def make(cost):
        def ctor(scenarios, stream=None):
            b = FakeBatch(scenarios, stream, cost)
            made.append(b)
            return b
        monkeypatch.setattr(P, "Batch", ctor)
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "fake-gpu")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return make, made, tmp_path


def costs(fastest):
    # every candidate costs 3 units except `fastest` (1 unit)
    return {c: (1.0 if c == fastest else 3.0) for c in autotune.CANDIDATES}


def scenarios(n=6, side=128):
    return [WL.Scenario(side, side, WL.ACO, 200, 8, 10 + i, 100, name=f"s{i}") for i in range(n)]


def test_picks_the_fastest_candidate_and_caches_it(fake_env):
    make, made, tmp = fake_env
    target = autotune.CANDIDATES[3]
    make(costs(target))
    scs = scenarios()
    assert autotune.tune(scs, steps=32, repeats=2) == target
    assert len(made) == 1 and made[0].closed           # one scratch batch, closed
    cache = json.loads((tmp / "autotune.json").read_text())
    (key, entry), = cache.items()
    assert key == f"fake-gpu|{autotune.size_class(scs)}"
    assert tuple(entry["choice"]) == target
    assert len(entry["timings_s"]) == len(autotune.CANDIDATES)
    # a second call with the same size class is answered from the cache
    make(costs(autotune.CANDIDATES[0]))
    assert autotune.tune(scs, steps=32, repeats=2) == target
    assert len(made) == 1


def test_without_cache_nothing_is_stored(fake_env):
    make, made, tmp = fake_env
    target = autotune.CANDIDATES[0]
    make(costs(target))
    assert autotune.tune(scenarios(), steps=32, repeats=2, use_cache=False) == target
    assert not (tmp / "autotune.json").exists()


def test_apply_sets_tiling_only_for_tiled_variants():
    b = FakeBatch([], cost={})
    for cand in autotune.CANDIDATES:
        b.calls.clear()
        autotune.apply(b, cand)
        variant, tw, th, cps = cand
        assert b.calls[0] == ("variant", variant)
        if variant in (P.VARIANT_AGENT, P.VARIANT_DEFERRED):
            assert len(b.calls) == 1
        else:
            assert b.calls[1] == ("tiling", tw, th, cps)


def test_size_class_separates_batches_that_differ():
    small, large = scenarios(6, 128), scenarios(6, 1024)
    assert autotune.size_class(small) != autotune.size_class(large)
    assert autotune.size_class(small) != autotune.size_class(scenarios(40, 128))
    assert autotune.size_class(small) == autotune.size_class(scenarios(6, 128))
    lem = [s.with_(model=WL.LEM) for s in small]
    assert autotune.size_class(small) != autotune.size_class(lem)
