"""Serving loop over the device-resident scenario pool (``sim_pool_*``).

Continuous batching: requests arrive over time (``workloads.Request``);
whenever the pool's HBM budget and slot count allow, waiting requests are
admitted in arrival order as slots; all live slots advance together in
chunks of ``chunk`` steps (one batched launch per step inside the library);
a slot that reaches its step count is read back and released, which frees
its memory for the next waiting request.  A request's result does not depend
on what else is in the pool: every random number is keyed by the request's
own seed, cell and step.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import pedsim as P


@dataclass
class Result:
    index: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    stats: dict
    grid: dict | None = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclass
class ServingReport:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    cell_updates: int = 0
    max_live: int = 0
    rejected_waits: int = 0

    def percentile(self, q: float) -> float:
        lat = np.array([r.latency_s for r in self.results])
        return float(np.percentile(lat, q)) if len(lat) else float("nan")

    def summary(self) -> dict:
        n = len(self.results)
        return {"requests": n, "p50_s": self.percentile(50), "p99_s": self.percentile(99),
                "scenarios_per_s": n / self.wall_s if self.wall_s else 0.0,
                "cell_updates_per_s": self.cell_updates / self.wall_s if self.wall_s else 0.0,
                "max_live_slots": self.max_live}


class ServingLoop:
    """Admits, steps and retires scenario requests on one GPU."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256, chunk: int = 16,
                 stream=None, keep_grids: bool = False):
        self.pool = P.Pool(hbm_budget_bytes, max_slots, stream=stream)
        self.chunk = chunk
        self.keep_grids = keep_grids

    def close(self) -> None:
        self.pool.close()

    def run(self, requests, realtime: bool = True) -> ServingReport:
        """Serves `requests` (sorted by arrival).  With realtime=True arrivals
        follow the wall clock from the call; otherwise every request counts as
        arrived at once (throughput mode)."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        live = {}  # slot -> (request, admitted time)
        rep = ServingReport()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or live:
            # admit in arrival order while the budget allows
            while pending and (not realtime or pending[0].arrival_s <= now()):
                slot = self.pool.admit(pending[0].scenario)
                if slot is None:
                    rep.rejected_waits += 1
                    break
                live[slot] = (pending.pop(0), now())
            rep.max_live = max(rep.max_live, len(live))
            if not live:
                if pending and realtime:
                    time.sleep(max(0.0, pending[0].arrival_s - now()))
                continue
            self.pool.step(self.chunk)
            for slot in self.pool.finished():
                req, adm = live.pop(slot)
                sc = req.scenario
                grid = self.pool.read_grid(slot, sc.W, sc.H) if self.keep_grids else None
                stats = self.pool.stats(slot)
                rep.results.append(Result(req.index, req.arrival_s if realtime else 0.0, adm, now(),
                                          stats, grid))
                rep.cell_updates += sc.cells * sc.steps
                self.pool.release(slot)
        rep.wall_s = now()
        rep.results.sort(key=lambda r: r.index)
        return rep
