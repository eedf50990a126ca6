"""Domain decomposition on the GPU: one grid advanced as column strips (each
strip stepped by sim_step_strip through the C ABI, halos of three columns
exchanged between steps) equals the CPU oracle's run of the whole grid bit
for bit -- occupancy, ids, both pheromone planes as raw bits, per-agent
arrival steps and tour lengths, and the moved / conflict / crossing
counters summed over the strips.  The strips live on one GPU here; the
exchange is the same code that moves halos between ranks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_4933_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_4933_gb300 import pedsim as P  # noqa: E402
from paper_1412_4933_gb300 import domain as D  # noqa: E402


def start(sc, n_strips):
    """The library's own placement of the scenario, loaded into strips."""
    sim = P.Sim(sc.W, sc.H, P.params_of(sc))
    sim.place(sc.seed)
    grid, agents = sim.read_grid(), sim.read_agents()
    sim.close()
    dom = D.StripDomain(sc.W, sc.H, P.params_of(sc), sc.seed, n_strips)
    dom.load(0, grid, agents)
    return dom


def same(label, dom, orc, aco):
    g, o, a = dom.read_grid(), orc.state(), dom.read_agents()
    assert np.array_equal(g["occ"], o["occ"]), f"{label}: occupancy"
    assert np.array_equal(g["ids"], o["ids"]), f"{label}: ids"
    if aco:
        assert np.array_equal(g["tauA"].view(np.uint32), o["tauA"].view(np.uint32)), f"{label}: tauA"
        assert np.array_equal(g["tauB"].view(np.uint32), o["tauB"].view(np.uint32)), f"{label}: tauB"
    # per-agent entries of the agents on the grid, taken from their strips
    assert np.array_equal(a["arrival"][1:], o["arrival"][1:]), f"{label}: arrival"
    assert np.array_equal(a["tour"][1:].view(np.uint32), o["tour"][1:].view(np.uint32)), \
        f"{label}: tour"
    c, s = dom.counters(), orc.stats()
    assert (c["moved"], c["conflicts"], c["crossed"]) == (s["moved"], s["conflicts"], s["crossed"]), \
        f"{label}: counters {c} vs {s}"


CASES = [
    # narrow strips, dense bands: agents cross strip boundaries all the time
    (WL.Scenario(48, 32, WL.ACO, 300, 16, 51, 60, rho=0.07, deposit_mode=1,
                 name="aco_48x32_three_strips_of_16"), 3),
    (WL.Scenario(48, 32, WL.LEM, 300, 16, 52, 60, name="lem_48x32_three_strips"), 3),
    (WL.Scenario(176, 80, WL.ACO, 1500, 30, 53, 90, rho=0.1, name="aco_176x80_ragged_two_strips"), 2),
    (WL.Scenario(176, 80, WL.ACO, 1500, 30, 54, 90, rho=0.1, alpha=2, beta=3,
                 name="aco_176x80_four_strips_alpha2_beta3"), 4),
]


@pytest.mark.parametrize("sc,n", CASES, ids=lambda c: c.name if hasattr(c, "name") else str(c))
def test_strips_match_the_whole_grid_every_step(sc, n):
    dom = start(sc, n)
    orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
    aco = sc.model == WL.ACO
    for t in range(sc.steps):
        dom.step(1)
        orc.step(1)
        same(f"{sc.name} step {t + 1}", dom, orc, aco)


def test_headline_workload_in_two_strips():
    """The 100K-agent 2048^2 ACO workload as two 1024-column strips, 120
    steps (the bands empty into the middle, where the strips meet)."""
    sc = WL.ACO_2048
    dom = start(sc, 2)
    orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
    done = 0
    for target in (1, 40, 120):
        dom.step(target - done)
        orc.step(target - done)
        done = target
        same(f"{sc.name} two strips, step {target}", dom, orc, True)


def test_strip_entry_point_rejects_bad_arguments():
    sc = CASES[0][0]
    prm = P.params_of(sc)
    lay = D.StripLayout(sc.W, 16, 32)
    st = D.StripState(torch, lay, sc.H, sc.agents, True, "cuda:0")
    args = (st.occ[0], st.occ[1], st.ids, st.tau[0][0], st.tau[1][0], st.tau[0][1], st.tau[1][1],
            st.arrival, st.tour, st.scratch, st.counters)
    ok = P.step_strip(lay.width, sc.H, lay.ea, sc.W, lay.lo, lay.hi, prm, 1, 0, *args)
    assert ok == P.OK
    torch.cuda.synchronize()
    # columns beyond the grid, an inverted interior, occupancy in == out
    assert P.step_strip(lay.width, sc.H, sc.W - 4, sc.W, lay.lo, lay.hi, prm, 1, 0, *args) == P.EINVAL
    assert P.step_strip(lay.width, sc.H, lay.ea, sc.W, 10, 5, prm, 1, 0, *args) == P.EINVAL
    bad = list(args)
    bad[1] = bad[0]
    assert P.step_strip(lay.width, sc.H, lay.ea, sc.W, lay.lo, lay.hi, prm, 1, 0, *bad) == P.EINVAL
