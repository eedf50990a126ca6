"""Serving pool and batched runner on the GPU: admission by HBM budget,
continuous batching, and every request's result equal to running it alone
(bit for bit); the autotuner's choice never changes results."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_4933_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_4933_gb300 import pedsim as P  # noqa: E402
from paper_1412_4933_gb300 import serving, autotune  # noqa: E402


def _alone(sc):
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    sim.place(sc.seed)
    sim.step(sc.steps)
    out = sim.read_grid(), sim.stats()
    sim.close()
    return out


def _same_grid(a, b, aco):
    assert np.array_equal(a["occ"], b["occ"])
    assert np.array_equal(a["ids"], b["ids"])
    if aco:
        assert np.array_equal(a["tauA"].view(np.uint32), b["tauA"].view(np.uint32))
        assert np.array_equal(a["tauB"].view(np.uint32), b["tauB"].view(np.uint32))


def test_serving_results_equal_running_alone():
    reqs = WL.serving_requests(14, rate_per_s=400.0, agents_lo=500, agents_hi=6000,
                               steps_lo=20, steps_hi=90)
    need = max(P.device_bytes(r.scenario.W, r.scenario.H, P.params_of(r.scenario)) for r in reqs)
    loop = serving.ServingLoop(hbm_budget_bytes=3 * need, max_slots=8, chunk=7, keep_grids=True)
    rep = loop.run(reqs, realtime=False)  # all waiting at once: the budget decides
    loop.close()
    assert len(rep.results) == len(reqs)
    assert rep.max_live >= 2            # requests overlapped on the device
    assert rep.rejected_waits > 0       # the budget made later requests wait
    for res, req in zip(rep.results, reqs):
        g, st = _alone(req.scenario)
        _same_grid(res.grid, g, req.scenario.model == WL.ACO)
        assert res.stats == st
    s = rep.summary()
    assert s["p99_s"] >= s["p50_s"] > 0


def test_serving_realtime_poisson_arrivals():
    reqs = WL.serving_requests(10, rate_per_s=200.0, agents_lo=500, agents_hi=4000,
                               steps_lo=20, steps_hi=60)
    loop = serving.ServingLoop(hbm_budget_bytes=1 << 30, max_slots=16, chunk=8)
    rep = loop.run(reqs)
    loop.close()
    assert [r.index for r in rep.results] == list(range(10))
    for res, req in zip(rep.results, reqs):
        assert res.finished_s >= req.arrival_s
        assert res.stats["step"] == req.scenario.steps


def test_pool_admission_by_budget():
    sc = WL.Scenario(64, 64, WL.ACO, 200, 8, 3, 30)
    need = P.device_bytes(64, 64, P.params_of(sc))
    pool = P.Pool(2 * need + 1, 8)
    a, b = pool.admit(sc), pool.admit(sc.with_(seed=4))
    assert a is not None and b is not None
    assert pool.admit(sc.with_(seed=5)) is None      # over budget: nothing allocated
    assert pool.bytes_in_use == 2 * need and pool.live == 2
    pool.step(30)
    assert sorted(pool.finished()) == sorted([a, b])
    pool.release(a)
    c = pool.admit(sc.with_(seed=5))                 # freed memory is reusable
    assert c is not None and pool.live == 2
    orc = O.Oracle(64, 64, O.make_params(**sc.params()), 4)
    orc.step(30)
    assert pool.stats(b) == orc.stats()
    pool.close()


@pytest.mark.parametrize("choice", autotune.CANDIDATES, ids=lambda c: f"v{c[0]}_{c[1]}x{c[2]}_c{c[3]}")
def test_every_batched_launch_configuration_is_bit_identical(choice):
    scs = WL.batched_scenarios(count=10, steps=25, side_lo=64, side_hi=320)
    batch = P.Batch(scs)
    autotune.apply(batch, choice)
    batch.step(25)
    for i, sc in enumerate(scs):
        orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
        orc.step(25)
        g, o = batch.read_grid(i), orc.state()
        _same_grid(g, o, sc.model == WL.ACO)
        assert batch.stats(i) == orc.stats()
    batch.close()


def test_autotuner_picks_a_candidate():
    scs = WL.batched_scenarios(count=16, steps=10, side_lo=128, side_hi=512)
    best = autotune.tune(scs, steps=8, use_cache=False)
    assert best in autotune.CANDIDATES
