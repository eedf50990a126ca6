"""The oracle and the study set-up against the values the paper prints
(fixtures under tests/golden/, each with its citation)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_4933_gb300 import study
from paper_1412_4933_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_fig2_sample_environment_placement(seed):
    """Sec. IV.a / Fig. 2: 16x16, 3-wide bands, 58 agents labelled 1 and 2,
    index numbers 1 .. 58 on the occupied cells."""
    g = _load("paper_fig2_environment.json")
    W, H, band, n = g["W"], g["H"], g["band"], g["agents_total"]
    o = O.Oracle(W, H, O.make_params(model=0, n_per_side=n // 2, band_cols=band), seed)
    st = o.state()
    occ, ids = st["occ"], st["ids"]
    occupied = occ > 0
    assert int(occupied.sum()) == n
    assert sorted(ids[occupied].tolist()) == list(range(1, n + 1))
    assert set(np.unique(occ[occupied]).tolist()) == set(g["labels"])
    cols1 = np.where(occ == 1)[1]
    cols2 = np.where(occ == 2)[1]
    assert cols1.min() >= 0 and cols1.max() < band
    assert cols2.min() >= W - band and cols2.max() < W
    assert int((occ == 1).sum()) == int((occ == 2).sum()) == n // 2


@pytest.mark.parametrize("group", [1, 2])
def test_fig2_crossing_line(group):
    """Sec. VI: in the 16x16 sample with 3-wide bands an agent has crossed on
    reaching the 14th line counted from its own side.  A lone walker from
    its own edge arrives exactly when it enters that line."""
    g = _load("paper_fig2_environment.json")
    W, H, band = g["W"], g["H"], g["band"]
    line = g["crossing_line_1_indexed"] - 1  # 0-based, counted from the walker's side
    occ = np.zeros((H, W), np.uint8)
    ids = np.zeros((H, W), np.uint32)
    x0 = 0 if group == 1 else W - 1
    occ[5, x0] = group
    ids[5, x0] = 1
    p = O.make_params(model=0, n_per_side=1, band_cols=band)
    o = O.Oracle(W, H, p, 9, state={"occ": occ, "ids": ids})
    arrival = None
    for t in range(1, W + 2):
        o.step(1)
        st = o.state()
        x = int(np.where(st["ids"][5] == 1)[0][0])
        from_own_side = x if group == 1 else W - 1 - x
        if arrival is None and st["arrival"][1] != 0:
            arrival = int(st["arrival"][1])
            assert from_own_side == line, (t, x)
    assert arrival == line  # one cell per step from line 0


def test_throughput_study_matches_paper_setup():
    """Sec. VI: the study's populations, repeats, steps and grid."""
    g = _load("paper_throughput_study.json")
    scs = study.study_scenarios()
    assert all(s.W == s.H == g["side"] for s in scs)
    assert all(s.steps == g["steps"] for s in scs)
    for model in (WL.LEM, WL.ACO):
        pops = sorted({s.agents for s in scs if s.model == model})
        assert pops == [g["first_total"] + k * g["increment"] for k in range(g["populations"])]
        for a in pops:
            runs = [s for s in scs if s.model == model and s.agents == a]
            assert len(runs) == g["repeats"]
            assert len({s.seed for s in runs}) == g["repeats"]
            assert all(s.n_per_side * 2 == a for s in runs)
