"""Seeded synthetic workloads (scenario descriptions only).

This module describes WHAT to simulate: grid sizes, agent counts, models,
evaporation rates, seeds and step counts of the synthetic scenarios that stand
in for the paper's 480x480 grid with 2K-100K agents in edge bands (Sec. III,
Sec. V).  It holds none of the automaton's arithmetic: placement and every
random number the method draws come from each side's own Philox4x64-10,
keyed by the scenario seed.  Both the CUDA path and the CPU oracle read their
scenario descriptions from here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace

import numpy as np

LEM, ACO = 0, 1


@dataclass(frozen=True)
class Scenario:
    W: int
    H: int
    model: int
    n_per_side: int
    band_cols: int
    seed: int
    steps: int
    rho: float = 0.05
    tau0: float = 1.0
    deposit: float = 1.0
    alpha: int = 1
    beta: int = 1
    deposit_mode: int = 0
    lem_sigma: float = 1.0
    name: str = ""

    @property
    def cells(self) -> int:
        return self.W * self.H

    @property
    def agents(self) -> int:
        return 2 * self.n_per_side

    def params(self) -> dict:
        d = asdict(self)
        for k in ("W", "H", "seed", "steps", "name"):
            d.pop(k)
        return d

    def with_(self, **kw) -> "Scenario":
        return replace(self, **kw)


# Single-scenario workloads: LEM 256^2, ACO 512^2, ACO 2048^2 (the 100K-agent
# roofline case) and an 8192^2 probe at the same density whose planes exceed
# the 129 MB L2.
LEM_256 = Scenario(256, 256, LEM, 1000, 16, 1, 500, name="lem_256x256_2k_agents")
ACO_512 = Scenario(512, 512, ACO, 5000, 32, 2, 1000, rho=0.05,
                   name="aco_512x512_10k_agents")
ACO_2048 = Scenario(2048, 2048, ACO, 50000, 64, 3, 2000, rho=0.02,
                    name="aco_2048x2048_100k_agents")
ACO_8192 = Scenario(8192, 8192, ACO, 800000, 256, 4, 200, rho=0.02,
                    name="aco_8192x8192_1.6m_agents_probe")

SINGLE = {s.name: s for s in (LEM_256, ACO_512, ACO_2048, ACO_8192)}


def round16(v: float) -> int:
    return max(16, int(round(v / 16.0)) * 16)


def band_for(n_per_side: int, H: int) -> int:
    """Placement band width: at most half of the band's cells are filled."""
    return max(1, math.ceil(n_per_side / (0.5 * H)))


def batched_scenarios(count: int = 256, steps: int = 500, first_seed: int = 1000,
                      gen_seed: int = 12345, side_lo: int = 128, side_hi: int = 1024):
    """Uneven batch: side log-uniform in [side_lo, side_hi] (rounded to 16),
    density uniform 2-30 %, split evenly between the groups, LEM or ACO by a
    fair coin, rho uniform 0.01-0.1 for ACO, seeds first_seed + i."""
    rng = np.random.default_rng(gen_seed)
    out = []
    ratio = side_hi / side_lo
    for i in range(count):
        side = round16(side_lo * ratio ** rng.uniform())
        side = min(max(side, side_lo), side_hi)
        density = rng.uniform(0.02, 0.30)
        model = ACO if rng.uniform() < 0.5 else LEM
        rho = float(np.float32(rng.uniform(0.01, 0.1)))
        n = int(round(density * side * side / 2))
        band = band_for(n, side)
        out.append(Scenario(side, side, model, n, band, first_seed + i, steps,
                            rho=rho if model == ACO else 0.05,
                            name=f"batch{i}"))
    return out


@dataclass(frozen=True)
class Request:
    index: int
    arrival_s: float
    scenario: Scenario


def serving_requests(count: int, rate_per_s: float = 200.0, arrival_seed: int = 7,
                     first_seed: int = 2000, agents_lo: int = 2000,
                     agents_hi: int = 100000, steps_lo: int = 200, steps_hi: int = 2000):
    """Poisson arrivals of scenario requests: total agents log-uniform in
    [agents_lo, agents_hi], density uniform 5-25 % on a square grid, LEM or
    ACO by a fair coin, rho uniform 0.01-0.1, steps uniform integers."""
    rng = np.random.default_rng(arrival_seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        n_total = agents_lo * (agents_hi / agents_lo) ** rng.uniform()
        density = rng.uniform(0.05, 0.25)
        side = round16(math.ceil(math.sqrt(n_total / density)))
        model = ACO if rng.uniform() < 0.5 else LEM
        rho = float(np.float32(rng.uniform(0.01, 0.1)))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        n = int(round(n_total / 2))
        band = band_for(n, side)
        out.append(Request(i, t, Scenario(side, side, model, n, band, first_seed + i, steps,
                                          rho=rho if model == ACO else 0.05,
                                          name=f"req{i}")))
    return out


def random_occupancy(W: int, H: int, density: float, seed: int):
    """A random grid state for rule tests: each cell holds an agent with the
    given probability, of either group; ids are a random permutation."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((H, W), np.uint8)
    filled = rng.uniform(size=(H, W)) < density
    occ[filled] = rng.integers(1, 3, size=int(filled.sum()), dtype=np.uint8)
    ids = np.zeros((H, W), np.uint32)
    n = int(filled.sum())
    ids[filled] = rng.permutation(n).astype(np.uint32) + 1
    return occ, ids


def shard(items, rank: int, world: int):
    """Independent scenarios split across ranks round-robin (no exchange is
    needed: every scenario's result depends on its own seed only)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(items)[rank::world]
