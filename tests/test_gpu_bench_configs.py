"""Parity at the configurations the benchmark times: bit-exact agreement
with the CPU oracle (tolerance 0) for

  * a sample of the benchmark's own 256-scenario batch (the largest grids of
    both models, the densest scenarios and the first few) over its full 500
    steps, run in the batch through the launch configuration the autotuner
    chooses for it, as the benchmark runs it;
  * the largest (97,884 agents) and the longest (1,992 steps) requests of the
    benchmark's serving stream, served through the continuous-batching loop
    together with other requests;
  * the 8192 x 8192 probe with 1.6M agents after the benchmark's warm-up and
    timed steps.

The oracle runs in spawned worker processes (one scenario each)."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1412_4933_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_4933_gb300 import pedsim as P  # noqa: E402
from paper_1412_4933_gb300 import autotune, serving  # noqa: E402


def oracle_final(W, H, params, seed, steps):
    """The oracle's state and counters after `steps` steps (worker process)."""
    from oracle import oracle as O
    o = O.Oracle(W, H, O.make_params(**params), seed)
    o.step(steps)
    st = o.state()
    return {k: st[k] for k in ("occ", "ids", "tauA", "tauB")}, o.stats()


@pytest.fixture(scope="module")
def workers():
    n = max(1, min(8, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        yield ex


def submit(workers, sc, steps):
    return workers.submit(oracle_final, sc.W, sc.H, sc.params(), sc.seed, steps)


def same(label, g, st, ref, aco):
    o, ost = ref
    assert np.array_equal(g["occ"], o["occ"]), f"{label}: occupancy"
    assert np.array_equal(g["ids"], o["ids"]), f"{label}: ids"
    if aco:
        assert np.array_equal(g["tauA"].view(np.uint32), o["tauA"].view(np.uint32)), f"{label}: tauA"
        assert np.array_equal(g["tauB"].view(np.uint32), o["tauB"].view(np.uint32)), f"{label}: tauB"
    assert st == ost, f"{label}: counters"


def batch_sample(scs):
    """Indices of the largest grid of each model, the densest scenario of
    each model and the first four."""
    pick = set(range(4))
    for model in (WL.LEM, WL.ACO):
        idx = [i for i, s in enumerate(scs) if s.model == model]
        pick.add(max(idx, key=lambda i: (scs[i].W, scs[i].agents)))
        pick.add(max(idx, key=lambda i: scs[i].agents / scs[i].cells))
    return sorted(pick)


def test_benchmark_batch_sample_full_run(workers):
    scs = WL.batched_scenarios(count=256, steps=500)
    sample = batch_sample(scs)
    futs = {i: submit(workers, scs[i], 500) for i in sample}
    choice = autotune.tune(scs)  # the benchmark's own call (cached per GPU and size class)
    batch = P.Batch(scs)
    autotune.apply(batch, choice)
    batch.step(500)
    assert batch.device_status() == 0
    assert max(scs[i].W for i in sample) == max(s.W for s in scs)
    for i in sample:
        sc = scs[i]
        same(f"{sc.name} ({sc.W}^2, {sc.agents} agents, choice {choice})", batch.read_grid(i),
             batch.stats(i), futs[i].result(timeout=900), sc.model == WL.ACO)
    batch.close()


def test_benchmark_serving_largest_and_longest_requests(workers):
    reqs = WL.serving_requests(200)
    big = max(reqs, key=lambda r: r.scenario.agents)
    long_ = max(reqs, key=lambda r: r.scenario.steps)
    assert big.scenario.agents > 95_000 and long_.scenario.steps > 1_950
    mix = [big, long_] + [r for r in reqs[:12] if r.scenario.agents < 20_000][:6]
    futs = {r.index: submit(workers, r.scenario, r.scenario.steps) for r in (big, long_)}
    free, _ = torch.cuda.mem_get_info()
    loop = serving.ServingLoop(int(free * 0.5), 512, chunk=16, keep_grids=True)
    rep = loop.run(mix, realtime=False)
    loop.close()
    assert rep.max_live >= 2
    by_index = {res.index: res for res in rep.results}
    for r in (big, long_):
        sc, res = r.scenario, by_index[r.index]
        same(f"request {r.index} ({sc.W}^2, {sc.agents} agents, {sc.steps} steps)", res.grid,
             res.stats, futs[r.index].result(timeout=900), sc.model == WL.ACO)


def test_hbm_probe_workload(workers):
    """The 8192^2 probe: placement, the benchmark's 16 warm-up and 20 timed
    steps (36 in all), in the library's default variant."""
    sc = WL.ACO_8192
    fut = submit(workers, sc, 36)
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    sim.place(sc.seed)
    sim.step(16)
    sim.step(20)
    g = sim.read_grid()
    same(sc.name, g, sim.stats(), fut.result(timeout=900), True)
    assert sim.device_status() == 0
    sim.close()
