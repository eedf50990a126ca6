"""Host logic of the continuous-batching serving loop, on the CPU: a fake
pool stands in for ``sim_pool_*`` (the GPU tests run the real one), so the
admission order, the waits when the pool is full, retirement and the report
are checked without a device."""
import time

import pytest

from paper_1412_4933_gb300 import serving, workloads as WL


class FakePool:
    """Slots that finish after their scenario's step count; at most
    `capacity` live at once (admit returns None beyond it, as the real pool
    does when its HBM budget or slot count is exhausted)."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.live = {}        # slot -> [scenario, steps done]
        self.admitted = []    # scenario names in admission order
        self.max_live = 0
        self.steps_issued = 0
        self.next_slot = 0

    def admit(self, sc):
        if len(self.live) >= self.capacity:
            return None
        slot = self.next_slot
        self.next_slot += 1
        self.live[slot] = [sc, 0]
        self.admitted.append(sc.name)
        self.max_live = max(self.max_live, len(self.live))
        return slot

    def step(self, n):
        self.steps_issued += n
        for entry in self.live.values():
            entry[1] = min(entry[0].steps, entry[1] + n)

    def finished(self):
        return [s for s, (sc, done) in self.live.items() if done >= sc.steps]

    def stats(self, slot):
        sc, done = self.live[slot]
        return {"step": done, "moved": 0}

    def read_grid(self, slot, W, H):
        return {"occ": None}

    def release(self, slot):
        del self.live[slot]

    def close(self):
        pass


def make_loop(pool, chunk=16, keep_grids=False):
    loop = serving.ServingLoop.__new__(serving.ServingLoop)
    loop.pool, loop.chunk, loop.keep_grids = pool, chunk, keep_grids
    return loop


def requests(n, steps=(40, 100)):
    """n requests arriving 1 ms apart, small scenarios, varied step counts."""
    out = []
    for i in range(n):
        sc = WL.Scenario(64, 64, WL.LEM, 100, 8, 100 + i, steps[i % len(steps)],
                         name=f"r{i}")
        out.append(WL.Request(i, 0.001 * i, sc))
    return out


def test_throughput_mode_serves_everything_in_arrival_order():
    pool = FakePool(capacity=3)
    reqs = requests(10)
    rep = make_loop(pool).run(reversed(reqs), realtime=False)  # unsorted input
    assert [r.index for r in rep.results] == list(range(10))
    assert pool.admitted == [f"r{i}" for i in range(10)]       # FIFO admission
    assert pool.max_live == 3 and rep.max_live == 3
    assert rep.rejected_waits > 0                              # the pool filled up
    assert rep.cell_updates == sum(r.scenario.cells * r.scenario.steps for r in reqs)
    for r in rep.results:
        assert r.stats["step"] == reqs[r.index].scenario.steps  # retired only when done
        assert r.finished_s >= r.admitted_s
    assert not pool.live                                        # every slot released


def test_a_slot_is_stepped_in_whole_chunks_until_its_last_step():
    pool = FakePool(capacity=1)
    reqs = [WL.Request(0, 0.0, WL.Scenario(64, 64, WL.LEM, 100, 8, 1, 50, name="a"))]
    make_loop(pool, chunk=16).run(reqs, realtime=False)
    assert pool.steps_issued == 64  # ceil(50 / 16) chunks of 16


def test_realtime_mode_waits_for_arrivals_and_reports_latency():
    pool = FakePool(capacity=8)
    reqs = [WL.Request(i, 0.02 * i, WL.Scenario(64, 64, WL.LEM, 100, 8, i, 16, name=f"q{i}"))
            for i in range(4)]
    t0 = time.perf_counter()
    rep = make_loop(pool).run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    assert wall >= 0.06 - 1e-3                  # the last request arrives at 60 ms
    assert len(rep.results) == 4
    for r in rep.results:
        assert r.admitted_s >= r.arrival_s - 1e-3  # never admitted before it arrived
        assert r.latency_s >= 0.0
    s = rep.summary()
    assert s["requests"] == 4 and s["p50_s"] <= s["p99_s"]
    assert s["scenarios_per_s"] == pytest.approx(4 / rep.wall_s)


def test_keep_grids_reads_each_result_back():
    pool = FakePool(capacity=2)
    rep = make_loop(pool, keep_grids=True).run(requests(3), realtime=False)
    assert all(r.grid is not None for r in rep.results)
