"""The paper's throughput study (Sec. VI) on the batched runner: scenario
construction and summary on CPU; a miniature study on the GPU whose every
scenario matches the oracle's counters exactly."""
import numpy as np
import pytest

from paper_1412_4933_gb300 import study as S
from paper_1412_4933_gb300 import workloads as WL


def test_study_scenarios_follow_the_paper_grid():
    scs = S.study_scenarios()
    assert len(scs) == 2 * 20 * 10
    assert {(s.W, s.H, s.steps) for s in scs} == {(480, 480, 25000)}
    agents = sorted({s.agents for s in scs})
    assert agents[0] == 2560 and agents[-1] == 51200 and np.all(np.diff(agents) == 2560)
    # bands hold each group at <= 90 % and never overlap; 3 columns at 1,280 per side
    for s in scs:
        assert s.n_per_side <= 0.9 * s.band_cols * s.H + 1e-9
        assert 2 * s.band_cols <= s.W
    assert min(s.band_cols for s in scs) == 3
    assert len({s.seed for s in scs}) == len(scs)
    # the library accepts every scenario (host-only validation)
    P = pytest.importorskip("paper_1412_4933_gb300.pedsim")
    assert all(P.validate(s.W, s.H, P.params_of(s)) == P.OK for s in scs[::37])


def test_summarize_means_and_checks():
    rows = []
    for model, vals in ((WL.LEM, [100, 150, 10]), (WL.ACO, [100, 200, 60])):
        for agents, v in zip((100, 200, 300), vals):
            for seed, dv in enumerate((-1, 1)):
                rows.append({"model": model, "agents": agents, "seed": seed, "crossed": v + dv})
    out = S.summarize(rows)
    means = {(t["model"], t["agents"]): t["crossed_mean"] for t in out["table"]}
    assert means[("LEM", 300)] == 10 and means[("ACO", 200)] == 200
    c = out["checks"]
    assert c["populations"] == 3 and c["aco_ge_lem_populations"] == 3
    assert c["populations_all_crossed_both"] == 1
    assert c["lem_peak_agents"] == 200 and c["aco_peak_agents"] == 200
    assert abs(c["aco_over_lem_total_gain"] - (360 / 260 - 1)) < 1e-12


@pytest.mark.gpu
def test_miniature_study_matches_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("needs a CUDA GPU")
    from oracle import oracle as O
    scs = S.study_scenarios(populations=3, seeds=2, steps=300, side=96, agents_step=256)
    rows, timing = S.run(scs, tune=False)
    assert timing["device_status"] == 0
    for sc, row in zip(scs, rows):
        orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
        orc.step(sc.steps)
        st = orc.stats()
        assert row["crossed"] == st["crossed"][0] + st["crossed"][1], sc.name
        assert row["moved"] == st["moved"], sc.name
