"""The paper's pedestrian-throughput study (Sec. V, Sec. VI) on the batched
runner.

Throughput is the number of pedestrians that cross to the opposite side
within a fixed number of steps (Sec. VI): here the count of agents whose
first entry into the opposite band is recorded (the `crossed` counters).
The study grid is 480 x 480; the population grows from 2,560 agents (1,280
per side) in steps of 2,560; every population runs for 25,000 steps with 10
seeds, for LEM and for ACO, and the crossed counts are averaged over the
seeds (Sec. VI).  The paper plots the first 20 populations (up to 51,200
agents), beyond which it reports gridlock.

Readings where the paper is silent: the start band is the narrowest one
that holds the group at no more than 90 % fill (3 columns for 1,280 agents
on 480 rows, the depth of the paper's Fig. 2a example); ACO uses the tour
deposit of Eq. 5 (the paper deposits by the agent's tour) with rho = 0.05,
tau0 = 1 and alpha = beta = 1.

    python -m paper_1412_4933_gb300.study --populations 20 --seeds 10 --steps 25000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as WL

SIDE = 480
AGENTS_STEP = 2560   # total agents added per population (Sec. VI)
BAND_FILL = 0.9


def study_scenarios(populations: int = 20, seeds: int = 10, steps: int = 25000, side: int = SIDE,
                    first_seed: int = 5000, rho: float = 0.05, models=(WL.LEM, WL.ACO),
                    agents_step: int = AGENTS_STEP):
    """Scenario list of the study: for each model, each population
    k = 1..populations (k * agents_step agents in total) and each seed."""
    out = []
    i = 0
    for model in models:
        for k in range(1, populations + 1):
            n = k * agents_step // 2
            band = max(1, math.ceil(n / (BAND_FILL * side)))
            for r in range(seeds):
                out.append(WL.Scenario(side, side, model, n, band, first_seed + i, steps,
                                       rho=rho if model == WL.ACO else 0.05,
                                       deposit_mode=1 if model == WL.ACO else 0,
                                       name=f"{'aco' if model == WL.ACO else 'lem'}_{2 * n}_s{r}"))
                i += 1
    return out


def summarize(rows):
    """Mean and standard deviation of the crossed count per (model,
    population), and the paper's qualitative statements checked on them."""
    groups = {}
    for r in rows:
        groups.setdefault((r["model"], r["agents"]), []).append(r["crossed"])
    table = []
    for (model, agents) in sorted(groups):
        v = np.array(groups[(model, agents)], dtype=np.float64)
        table.append({"model": "ACO" if model == WL.ACO else "LEM", "agents": agents,
                      "crossed_mean": float(v.mean()), "crossed_std": float(v.std()),
                      "runs": int(v.size)})
    by = {(t["model"], t["agents"]): t["crossed_mean"] for t in table}
    pops = sorted({t["agents"] for t in table})
    both = [a for a in pops if ("LEM", a) in by and ("ACO", a) in by]
    lem = np.array([by[("LEM", a)] for a in both])
    aco = np.array([by[("ACO", a)] for a in both])
    checks = {}
    if len(both):
        # overall gain of ACO over LEM across the populations (the paper: +39.6 %)
        checks["aco_over_lem_total_gain"] = float(aco.sum() / max(lem.sum(), 1.0) - 1.0)
        checks["aco_ge_lem_populations"] = int((aco >= lem).sum())
        checks["populations"] = len(both)
        # populations where both models move everyone across (low density)
        checks["populations_all_crossed_both"] = int(sum(
            1 for a, l, c in zip(both, lem, aco) if l >= a - 0.5 and c >= a - 0.5))
        # peak of each model (the paper: ACO peaks at 28,160 agents)
        checks["lem_peak_agents"] = int(both[int(np.argmax(lem))])
        checks["aco_peak_agents"] = int(both[int(np.argmax(aco))])
    return {"table": table, "checks": checks}


def run(scenarios, stream=None, variant=None, tune: bool = True):
    """Advances every scenario of the study in one batch and returns one row
    per scenario (model, agents, seed, crossed, moved)."""
    import torch
    from . import pedsim as P
    from . import autotune
    steps = scenarios[0].steps
    assert all(s.steps == steps for s in scenarios), "one step count per batch"
    b = P.Batch(scenarios, stream=stream)
    try:
        if variant is not None:
            b.set_variant(variant)
        elif tune:
            autotune.apply(b, autotune.tune(scenarios, stream=stream))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rows = []
        for i, sc in enumerate(scenarios):
            st = b.stats(i)
            rows.append({"model": sc.model, "agents": sc.agents, "seed": sc.seed,
                         "crossed": int(st["crossed"][0] + st["crossed"][1]),
                         "moved": int(st["moved"]), "name": sc.name})
        status = b.device_status()
    finally:
        b.close()
    cells = sum(s.cells for s in scenarios) * steps
    return rows, {"seconds": wall, "cell_updates_per_s": cells / wall, "device_status": status}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--populations", type=int, default=20)
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--steps", type=int, default=25000)
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--out", default=None, help="write rows, summary and timing as JSON")
    args = ap.parse_args()
    scs = study_scenarios(args.populations, args.seeds, args.steps, args.side)
    rows, timing = run(scs)
    result = {"config": vars(args), "timing": timing, **summarize(rows)}
    text = json.dumps(result, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(json.dumps({"timing": timing, "checks": result["checks"]}))


if __name__ == "__main__":
    main()
