"""GPU parity: the CUDA path through the C ABI equals the CPU oracle bit for
bit (tolerance 0: occupancy, ids, both pheromone planes as raw bits,
per-agent arrival and tour arrays, counters), at every step on small grids,
on the single-scenario workloads at full size, for every tile shape and
every step variant, on edge cases, after checkpoint/resume, and for batched
runs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_4933_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_4933_gb300 import pedsim as P  # noqa: E402

# Step variants that keep their own state between steps (the two-pass
# variant is the plain baseline and runs on the small grids only).
VARIANTS = [P.VARIANT_TILED, P.VARIANT_FUSED, P.VARIANT_AGENT, P.VARIANT_DEFERRED]
VARIANT_IDS = ["tiled", "fused", "agent", "deferred"]


def oparams(sc):
    return O.make_params(**sc.params())


def assert_same(sim, orc, label, aco=True, agents=True):
    g = sim.read_grid()
    o = orc.state()
    assert np.array_equal(g["occ"], o["occ"]), f"{label}: occupancy differs"
    assert np.array_equal(g["ids"], o["ids"]), f"{label}: ids differ"
    if aco:
        assert np.array_equal(g["tauA"].view(np.uint32), o["tauA"].view(np.uint32)), f"{label}: tauA"
        assert np.array_equal(g["tauB"].view(np.uint32), o["tauB"].view(np.uint32)), f"{label}: tauB"
    if agents:
        a = sim.read_agents()
        assert np.array_equal(a["arrival"], o["arrival"]), f"{label}: arrival"
        assert np.array_equal(a["tour"].view(np.uint32), o["tour"].view(np.uint32)), f"{label}: tour"


def make_pair(sc, variant=None, tiling=None):
    """The CUDA path (the library's default variant unless one is given)
    and the oracle, both placed with the scenario's seed."""
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    if variant is not None:
        sim.set_variant(variant)
    if tiling:
        sim.set_tiling(*tiling)
    sim.place(sc.seed)
    return sim, O.Oracle(sc.W, sc.H, oparams(sc), sc.seed)


SMALL = [
    WL.Scenario(64, 48, WL.LEM, 500, 20, 21, 120, name="lem_64x48_dense"),
    WL.Scenario(64, 48, WL.ACO, 500, 20, 22, 120, rho=0.05, name="aco_64x48_dense"),
    WL.Scenario(176, 80, WL.ACO, 1500, 30, 23, 80, rho=0.1, name="aco_176x80_ragged"),
    WL.Scenario(176, 80, WL.LEM, 1500, 30, 24, 80, name="lem_176x80_ragged"),
]


@pytest.mark.parametrize("sc", [WL.LEM_256, WL.ACO_512, WL.ACO_2048] + SMALL,
                         ids=lambda s: s.name)
def test_placement_matches_oracle(sc):
    sim, orc = make_pair(sc)
    assert_same(sim, orc, f"{sc.name} placement", aco=sc.model == WL.ACO)
    assert sim.stats() == orc.stats()


@pytest.mark.parametrize("variant", VARIANTS + [P.VARIANT_TWO_PASS],
                         ids=VARIANT_IDS + ["two_pass"])
@pytest.mark.parametrize("sc", SMALL, ids=lambda s: s.name)
def test_every_step_small(sc, variant):
    sim, orc = make_pair(sc, variant)
    aco = sc.model == WL.ACO
    for t in range(sc.steps):
        assert_same(sim, orc, f"{sc.name} step {t}", aco=aco, agents=(t % 10 == 0))
        sim.step(1)
        orc.step(1)
    assert_same(sim, orc, f"{sc.name} final", aco=aco)
    assert sim.stats() == orc.stats()
    assert sim.device_status() == 0


TILINGS = [(P.VARIANT_TILED, 128, 8), (P.VARIANT_TILED, 128, 16),
           (P.VARIANT_FUSED, 32, 16), (P.VARIANT_FUSED, 64, 8), (P.VARIANT_FUSED, 64, 16),
           (P.VARIANT_FUSED, 128, 8), (P.VARIANT_FUSED, 128, 16)]


@pytest.mark.parametrize("tiling", TILINGS, ids=lambda t: f"v{t[0]}_{t[1]}x{t[2]}")
def test_every_tile_shape(tiling):
    sc = SMALL[2]
    variant, tw, th = tiling
    sim, orc = make_pair(sc, variant=variant, tiling=(tw, th, 0))
    for t in range(40):
        sim.step(1)
        orc.step(1)
        assert_same(sim, orc, f"tile {tiling} step {t + 1}", agents=False)
    # graph replays (16 steps per graph) and a ragged remainder
    sim.step(37)
    orc.step(37)
    assert_same(sim, orc, f"tile {tiling} after graphs")
    assert sim.stats() == orc.stats()


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("sc", [WL.LEM_256, WL.ACO_512], ids=lambda s: s.name)
def test_workload_every_step(sc, variant):
    """Full step count; every step for the first 64, then every 16 (graph)."""
    sim, orc = make_pair(sc, variant)
    aco = sc.model == WL.ACO
    t = 0
    while t < sc.steps:
        n = 1 if t < 64 else min(16, sc.steps - t)
        sim.step(n)
        orc.step(n)
        t += n
        assert_same(sim, orc, f"{sc.name} step {t}", aco=aco, agents=(t % 64 == 0))
    assert_same(sim, orc, f"{sc.name} final", aco=aco)
    s_gpu, s_orc = sim.stats(), orc.stats()
    assert s_gpu == s_orc
    assert s_gpu["moved"] > 0


def test_aco_2048_full_run():
    """The 100K-agent ACO workload at full size for its full 2000 steps, in
    the launch configuration the benchmark times (the library's default
    variant, graph replays)."""
    sc = WL.ACO_2048
    sim, orc = make_pair(sc)
    done = 0
    for target in (1, 2, 16, 200, 1000, 2000):
        sim.step(target - done)
        orc.step(target - done)
        done = target
        assert_same(sim, orc, f"{sc.name} step {target}")
        assert sim.stats() == orc.stats()
    assert sim.device_status() == 0


def test_more_agent_blocks_than_one_wave():
    """400,000 agents (1,563 agent blocks): more proposal blocks than one
    resident wave of the first agent kernel holds, so the ones beyond the
    first wave are interleaved with the stream blocks; checked every step
    against the oracle, and over a graph replay of 16 steps."""
    sc = WL.Scenario(1024, 1024, WL.ACO, 200_000, 256, 31, 40, rho=0.05, deposit_mode=1,
                     name="aco_1024x1024_400k_agents")
    sim, orc = make_pair(sc)
    for t in range(1, 5):
        sim.step(1)
        orc.step(1)
        assert_same(sim, orc, f"{sc.name} step {t}")
    sim.step(16)
    orc.step(16)
    assert_same(sim, orc, f"{sc.name} step 20")
    assert sim.stats() == orc.stats()
    assert sim.device_status() == 0
    sim.close()


EDGE = [
    WL.Scenario(32, 16, WL.ACO, 0, 4, 1, 160, rho=0.5, name="empty_grid_decay_to_subnormal"),
    WL.Scenario(64, 32, WL.ACO, 8 * 32, 8, 2, 60, rho=0.05, name="full_bands"),
    WL.Scenario(16, 16, WL.LEM, 40, 4, 3, 60, name="minimal_16x16_lem"),
    WL.Scenario(16, 16, WL.ACO, 60, 8, 4, 60, rho=0.2, name="minimal_16x16_touching_bands"),
    WL.Scenario(96, 48, WL.ACO, 600, 24, 5, 80, rho=0.03, deposit_mode=1, name="deposit_inverse_tour"),
    WL.Scenario(96, 48, WL.ACO, 600, 24, 6, 80, rho=0.03, alpha=2, beta=0, name="alpha2_beta0"),
    WL.Scenario(96, 48, WL.ACO, 600, 24, 7, 80, rho=1.0, tau0=0.0, name="rho1_tau0_zero"),
    WL.Scenario(96, 48, WL.LEM, 600, 24, 8, 80, lem_sigma=2.0, name="lem_sigma2"),
    WL.Scenario(96, 48, WL.ACO, 600, 24, 9, 80, rho=0.05, alpha=4, beta=4, deposit=0.25,
                name="alpha4_beta4"),
]


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("sc", EDGE, ids=lambda s: s.name)
def test_edge_cases(sc, variant):
    sim, orc = make_pair(sc, variant)
    aco = sc.model == WL.ACO
    for t in range(sc.steps):
        sim.step(1)
        orc.step(1)
        assert_same(sim, orc, f"{sc.name} step {t + 1}", aco=aco, agents=(t % 8 == 0))
    assert sim.stats() == orc.stats()


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
def test_random_dense_states_one_step(model, variant):
    """Arbitrary dense states (including wall contact) loaded through
    sim_set_state; one step from each equals the oracle's."""
    rng = np.random.default_rng(17 + model)
    W, H = 48, 32
    prm = dict(model=model, band_cols=24, rho=0.07)
    for trial in range(40):
        occ, _ = WL.random_occupancy(W, H, rng.uniform(0.1, 0.8), 100 + trial)
        flat = occ.reshape(-1)
        nz = np.flatnonzero(flat)
        if len(nz) % 2:  # the ABI holds 2N agents
            flat[nz[-1]] = 0
            nz = nz[:-1]
        n = len(nz)
        ids = np.zeros((H, W), np.uint32)
        ids.reshape(-1)[nz] = rng.permutation(n).astype(np.uint32) + 1
        tauA = rng.uniform(0, 3, size=(H, W)).astype(np.float32)
        tauB = rng.uniform(0, 3, size=(H, W)).astype(np.float32)
        arrival = np.zeros(n + 1, np.uint32)
        step = int(rng.integers(0, 1000))
        seed = int(rng.integers(0, 2**63))
        sim = P.Sim(W, H, P.make_params(n_per_side=n // 2, **prm))
        sim.set_variant(variant)
        sim.set_state(seed, step, occ, ids, tauA, tauB, arrival)
        orc = O.Oracle(W, H, O.make_params(n_per_side=n // 2, **prm), seed,
                       state={"occ": occ, "ids": ids, "tauA": tauA, "tauB": tauB,
                              "arrival": arrival}, step=step)
        assert_same(sim, orc, f"trial {trial} loaded", aco=model == WL.ACO)
        for k in range(3):
            sim.step(1)
            orc.step(1)
            assert_same(sim, orc, f"trial {trial} step {k + 1}", aco=model == WL.ACO)


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("sc", [SMALL[1], EDGE[4]], ids=lambda s: s.name)
def test_checkpoint_resume_bit_exact(sc, variant):
    a, orc = make_pair(sc, variant)
    a.step(23)
    blob = a.save()
    a.step(41)
    b = P.Sim(sc.W, sc.H, P.params_of(sc))
    b.set_variant(variant)
    b.load(blob)
    b.step(41)
    orc.step(64)
    assert_same(a, orc, "uninterrupted")
    assert_same(b, orc, "resumed")
    assert a.stats() == b.stats() == orc.stats()


def test_launches_per_step_query():
    """sim_launches_per_step reports each variant's kernels of one step."""
    sc = SMALL[1]
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    try:
        for v, n in ((P.VARIANT_AGENT, 2), (P.VARIANT_FUSED, 2), (P.VARIANT_TILED, 3),
                     (P.VARIANT_TWO_PASS, 3), (P.VARIANT_DEFERRED, 2)):
            sim.set_variant(v)
            assert sim.launches_per_step() == n
    finally:
        sim.close()


def test_runs_on_a_side_stream():
    sc = SMALL[1]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=s)
        sim.place(sc.seed)
        sim.step(50)
    orc = O.Oracle(sc.W, sc.H, oparams(sc), sc.seed)
    orc.step(50)
    assert_same(sim, orc, "side stream")


def test_instances_in_turn_from_a_captured_graph():
    """The benchmark's launch configuration: instances stepped in turn, one
    step each, from a CUDA graph of several rounds captured around the
    library's launches and replayed; every instance matches the oracle."""
    scs = [SMALL[1], SMALL[1].with_(seed=SMALL[1].seed + 1), EDGE[4]]
    s = torch.cuda.Stream()
    sims = []
    with torch.cuda.stream(s):
        for sc in scs:
            sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=s)
            sim.place(sc.seed)
            sim.step(3)
            sims.append(sim)
    g = torch.cuda.CUDAGraph()
    # the host's copy of the step index counts the captured steps only (3 +
    # 3): the device's (3 + 12) has the other parity, so a read-back that
    # trusted the host copy would read the other pheromone plane
    rounds, replays = 3, 4
    with torch.cuda.graph(g, stream=s):
        for _ in range(rounds):
            for sim in sims:
                sim.step(1)
    with torch.cuda.stream(s):
        for _ in range(replays):
            g.replay()
    torch.cuda.synchronize()
    for sc, sim in zip(scs, sims):
        orc = O.Oracle(sc.W, sc.H, oparams(sc), sc.seed)
        orc.step(3 + rounds * replays)
        assert_same(sim, orc, f"{sc.name} after graph replays", aco=sc.model == WL.ACO)
        assert sim.stats() == orc.stats()
        assert sim.device_status() == 0
        sim.close()


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
def test_batch_matches_single_runs(variant):
    scs = WL.batched_scenarios(count=12, steps=40, side_lo=64, side_hi=256)
    batch = P.Batch(scs)
    batch.set_variant(variant)
    batch.step(3)
    batch.step(37)
    for i, sc in enumerate(scs):
        orc = O.Oracle(sc.W, sc.H, oparams(sc), sc.seed)
        orc.step(40)
        g, o = batch.read_grid(i), orc.state()
        assert np.array_equal(g["occ"], o["occ"]), sc
        assert np.array_equal(g["ids"], o["ids"]), sc
        if sc.model == WL.ACO:
            assert np.array_equal(g["tauA"].view(np.uint32), o["tauA"].view(np.uint32))
            assert np.array_equal(g["tauB"].view(np.uint32), o["tauB"].view(np.uint32))
        assert batch.stats(i) == orc.stats()
    assert batch.device_status() == 0


def test_variant_switch_mid_run():
    """Switching variants between steps continues the same trajectory (the
    agent variant rebuilds its positions from the planes)."""
    sc = SMALL[2]
    sim, orc = make_pair(sc, P.VARIANT_TILED)
    for v in (P.VARIANT_AGENT, P.VARIANT_FUSED, P.VARIANT_AGENT, P.VARIANT_DEFERRED,
              P.VARIANT_TILED, P.VARIANT_DEFERRED, P.VARIANT_AGENT, P.VARIANT_DEFERRED,
              P.VARIANT_FUSED):
        sim.set_variant(v)
        sim.step(13)
        orc.step(13)
        assert_same(sim, orc, f"after variant {v}")
    assert sim.stats() == orc.stats()


# --------------------------------------------------------------------------
# Deferred evaporation: values are brought up to date only where read and in
# a rolling refresh, so they must be compared after runs with no read-back
# in between (every read-back brings every cell up to date first).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sc", SMALL[1:3] + [EDGE[0], EDGE[4], EDGE[6], EDGE[8]],
                         ids=lambda s: s.name)
def test_deferred_sparse_read_back(sc):
    sim, orc = make_pair(sc, P.VARIANT_DEFERRED)
    done = 0
    # gaps shorter and longer than the 32-step refresh period, odd and even
    # end steps, plain launches and graph replays
    for gap in (1, 5, 31, 32, 33, 16, 47, 64, 3):
        sim.step(gap)
        orc.step(gap)
        done += gap
        assert_same(sim, orc, f"{sc.name} step {done}")
        assert sim.stats() == orc.stats()
    assert sim.device_status() == 0


def test_deferred_aco_2048_full_run():
    """The 100K-agent ACO workload for its full 2000 steps with deferred
    evaporation, compared at a few steps only (values age between them)."""
    sc = WL.ACO_2048
    sim, orc = make_pair(sc, P.VARIANT_DEFERRED)
    done = 0
    for target in (7, 40, 333, 1000, 2000):
        sim.step(target - done)
        orc.step(target - done)
        done = target
        assert_same(sim, orc, f"{sc.name} deferred step {target}")
        assert sim.stats() == orc.stats()
    assert sim.device_status() == 0
    sim.close()


def test_deferred_rejects_tiling_and_reports_two_launches():
    sc = SMALL[1]
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    try:
        sim.set_variant(P.VARIANT_DEFERRED)
        assert sim.launches_per_step() == 2
        with pytest.raises(P.PedsimError):
            sim.set_tiling(64, 16, 0)
    finally:
        sim.close()
