"""Benchmark of the pedestrian-CA step on GB300.

Headline (one JSON line on rank 0): cell-updates/s of the ACO step on the
2048x2048 grid with 100K agents (50K per side in 64-column bands, rho 0.02),
one "step" = one synchronous automaton step (proposal, gather resolution,
move, evaporation + deposit, counters) over the whole grid, inputs resident
in HBM.  One scenario's working set (~92 MB) would stay in the 129 MB L2,
so the timed steps take inputs larger than L2: four resident instances of
the workload (seeds 3..6, each after --warmup untimed steps) are stepped in
turn, one single-scenario step each, so every step reads its state from HBM
and the write-backs of earlier steps land inside the timed region.  The K
timed steps are one CUDA graph of exactly K steps; after one untimed replay
it is replayed --repeats times, each replay timed with one event pair
between barriers, and the headline is the median region.

Also reported on the same line:
  flushed_per_step
                the same single-scenario step with the L2 flushed before
                each step (a 512 MB write, then a 256 MB read of another
                buffer, so the flush's own write-backs happen before the
                step) and an event pair around each step: every step then
                also starts with cold instruction and descriptor caches
  flushed_write_only
                the same with the write-only flush (its write-backs land
                in the step)
  roofline      the step's kernels (proposals + stream, resolution):
                algorithmic bytes (18 B/cell) / step time vs the measured HBM
                copy bandwidth
  cpu_baseline  the single-threaded CPU oracle on a bounded sample
  e2e           the same metric end to end through the C ABI with host
                buffers: H2D of the initial state (pinned), the scenario's
                2000 steps, D2H of the final grid and counters (one
                instance, its state L2-resident across the run; bytes per
                step = the run's bytes / 2000)
  deferred_evaporation
                the same workload and timing with the deferred-evaporation
                step (per-cell stamps, bit-identical results, 18/32 B per
                cell-step of dense traffic), reported beside the headline
  steady        steps replayed back to back (CUDA graph), no flush: the
                simulation's own L2-resident regime
  inputs_larger_than_l2
                four independent copies of the headline scenario advanced
                together (inputs 4 x 105 MiB > L2), graph replays timed with
                one event pair: the cold-L2 step without per-step events
  batched       256 uneven scenarios x 500 steps in batched launches (the
                autotuner's configuration), vs the same scenarios and steps
                run one scenario at a time; algorithmic GB/s beside it
  serving       Poisson request stream through the serving pool: p50/p99
  domain_strips the headline workload as two column strips on this GPU
                (per-strip step plus halo exchange between the strips),
                beside the single-grid step

`--impl reference` times the CPU oracle instead (the reference arm).
Under torchrun each rank runs an independent replica (no collective on the
data path; weak scaling); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1412_4933_gb300 import workloads as WL  # noqa: E402

L2_FLUSH_BYTES = 512 << 20
ROTATING_INSTANCES = 4  # headline: 4 x 105 MiB of state at 2048^2, well above the L2
NOMINAL_HBM_GBPS = 7900.0  # GB300 HBM3e nominal, for context beside the measured peak
ALGO_BYTES_PER_CELL = {WL.LEM: 2, WL.ACO: 18}
KERNEL_SOURCES = ["paper_1412_4933_gb300/csrc/pedsim_agent.cu",
                  "paper_1412_4933_gb300/csrc/pedsim_rules.cuh",
                  "paper_1412_4933_gb300/csrc/pedsim_ptx.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "agent_step_aco_2048x2048_traffic.md")
# Step variants selectable for the headline (the library default is agent),
# their kernels, and the kernels one sim_step(1) call launches: agent:
# proposals + stream, then resolution (which also advances the step index);
# tiled: proposals, resolution, step index; fused: one kernel + step index;
# two-pass: two kernels + step index.
VARIANTS = {"agent": lambda P: P.VARIANT_AGENT, "tiled": lambda P: P.VARIANT_TILED,
            "fused": lambda P: P.VARIANT_FUSED, "two_pass": lambda P: P.VARIANT_TWO_PASS,
            "deferred": lambda P: P.VARIANT_DEFERRED}
KERNEL_NAMES = {"agent": "agent_stage1_kernel + agent_resolve_kernel",
                "tiled": "propose_tile_kernel<16> + resolve_tile_kernel<16>",
                "fused": "fused_step_kernel<64,16>",
                "two_pass": "propose_plane_kernel + resolve_plane_kernel",
                "deferred": "deferred_stage1_kernel + deferred_resolve_kernel"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic():
    """Per-step DRAM bytes of the step's kernels from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    src = cur = None
    for line in text.splitlines():
        if line.startswith("kernel_source_sha256_16:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            cur = float(line.split(":", 1)[1].strip())
    return cur if (src == kernel_source_hash() and cur) else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self) -> dict:
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def max_over_ranks(v: float, dist, device=None) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# --------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and reference arm)
# --------------------------------------------------------------------------
def oracle_rate(sc, steps: int, warm: int = 0):
    """Cell-updates/s of the single-threaded oracle over `steps` steps of
    `sc` after placement and `warm` untimed steps."""
    from oracle import oracle as O
    orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
    if warm:
        orc.step(warm)
    t0 = time.perf_counter()
    orc.step(steps)
    dt = time.perf_counter() - t0
    return sc.cells * steps / dt, dt


def oracle_multicore(scs, steps: int, cores: int):
    """The oracle on `cores` host cores at once, one scenario per core (the
    first `cores` scenarios), `steps` steps each, in spawned processes:
    aggregate cell-updates/s over the wall time of the parallel run."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    jobs = scs[:cores]
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(O.timed_run, sc.W, sc.H, sc.params(), sc.seed, steps) for sc in jobs]
        res = [f.result(timeout=600) for f in futs]
    # the workers step at the same time, each timing its own steps (process
    # start-up and placement excluded): total work over the longest run
    work = sum(r[0] for r in res)
    longest = max(r[1] for r in res)
    return {"value": work / longest, "unit": "cell-updates/s", "cores": len(jobs), "kind": "oracle",
            "sample": f"{steps} steps of each of the first {len(jobs)} batch scenarios, one per "
                      f"core in parallel (longest {longest:.2f} s)"}


def run_reference(args, sc):
    world, rank, local, dist = dist_setup(args)
    if rank != 0:
        return 0
    from oracle import oracle as O
    orc = O.Oracle(sc.W, sc.H, O.make_params(**sc.params()), sc.seed)
    orc.step(args.warmup)
    t0 = time.perf_counter()
    orc.step(args.steps)
    dt = time.perf_counter() - t0
    value = sc.cells * args.steps / dt
    line = {
        "impl": "reference", "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sc.name, "W": sc.W, "H": sc.H, "agents": sc.agents,
                   "model": "ACO" if sc.model else "LEM", "rho": sc.rho, "seed": sc.seed,
                   "l2": "cpu"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps of {sc.name} after {args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def rotating_instances(P, torch, sc, stream, variant, warmup: int, count: int):
    """`count` resident instances of the workload (seeds sc.seed + k), each
    placed and advanced `warmup` steps."""
    sims = []
    with torch.cuda.stream(stream):
        for k in range(count):
            s = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
            s.set_variant(variant)
            s.place(sc.seed + k)
            s.step(warmup)
            sims.append(s)
    torch.cuda.synchronize()
    return sims


L2_BYTES = 129 << 20  # GB300 L2
HEADLINE_REPEATS = 5  # timed regions of exactly K steps each; the headline is their median


def rotating_l2_note(P, sc) -> str:
    """How the headline keeps its inputs out of L2, with the instances'
    actual device state (the library's own size query)."""
    each = P.device_bytes(sc.W, sc.H, P.params_of(sc))
    total = ROTATING_INSTANCES * each
    where = ("inputs larger than L2: every step reads its state from HBM" if total > L2_BYTES
             else "inputs fit in L2 together (this workload is launch-bound, not HBM-bound)")
    return (f"{where}; {ROTATING_INSTANCES} resident instances of the workload (seeds "
            f"{sc.seed}..{sc.seed + ROTATING_INSTANCES - 1}, {each / 2**20:.0f} MiB of device "
            f"state each, {total / 2**20:.0f} MiB in all against the {L2_BYTES >> 20} MiB L2) "
            f"stepped in turn, one step each, from one CUDA graph of exactly the timed steps; "
            f"one event pair around each replay")


def capture_steps(sims, torch, stream, steps: int):
    """One CUDA graph of exactly `steps` single-scenario steps, step i
    advancing instance i % len(sims) (the library's launches go into the
    capturing stream; consecutive kernels overlap by programmatic dependent
    launch inside the graph)."""
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for i in range(steps):
            sims[i % len(sims)].step(1)
    torch.cuda.synchronize()
    return g


def time_graph_repeats(graph, torch, stream, repeats: int, dist=None, device=None):
    """Replays `graph` once untimed (graph upload, more warm-up), then
    `repeats` times, each replay bracketed by a barrier, a device
    synchronisation and one CUDA-event pair on the launching stream.
    Returns the max-over-ranks seconds of each timed replay."""
    with torch.cuda.stream(stream):
        graph.replay()
    torch.cuda.synchronize()
    out = []
    for _ in range(repeats):
        barrier(dist, device)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(dist, device)
        out.append(max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, device))
    return out


def time_steps_flushed(sim, torch, stream, steps: int, flush):
    """Sum of per-step CUDA-event times; L2 flushed between steps (outside
    the events)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        flush()
        evs[i][0].record(stream)
        sim.step(1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in evs]


def e2e_run(P, torch, sc, stream, reps: int):
    """End to end through the C ABI from pinned host buffers: set the state,
    run the scenario's steps, read the final grid and counters back."""
    cells = sc.cells
    n = sc.agents
    # initial state from the library's own placement, staged in pinned memory
    probe = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
    probe.place(sc.seed)
    g0 = probe.read_grid()
    probe.close()
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    h_occ, h_ids = pin(cells, torch.uint8), pin(cells, torch.int32).view(np.uint32)
    h_ta, h_tb = pin(cells, torch.float32), pin(cells, torch.float32)
    h_arr = pin(n + 1, torch.int32).view(np.uint32)
    h_occ[:] = g0["occ"].reshape(-1); h_ids[:] = g0["ids"].reshape(-1)
    h_ta[:] = g0["tauA"].reshape(-1); h_tb[:] = g0["tauB"].reshape(-1); h_arr[:] = 0
    o_occ, o_ids = pin(cells, torch.uint8), pin(cells, torch.int32).view(np.uint32)
    o_ta, o_tb = pin(cells, torch.float32), pin(cells, torch.float32)
    sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
    aco = sc.model == WL.ACO
    h2d = cells * (1 + 4) + (8 * cells if aco else 0) + 4 * (n + 1)
    d2h = cells * (1 + 4) + (8 * cells if aco else 0) + 64
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_state(sc.seed, 0, h_occ, h_ids, h_ta if aco else None, h_tb if aco else None, h_arr)
        sim.step(sc.steps)
        P._lib.sim_read_grid(sim.handle, P._ptr(o_occ), P._ptr(o_ids),
                             P._ptr(o_ta) if aco else None, P._ptr(o_tb) if aco else None)
        st = sim.stats()
        dt = time.perf_counter() - t0
        if r > 0:  # first run is warm-up
            times.append(dt)
    sim.close()
    best = statistics.median(times)
    return {"value": sc.cells * sc.steps / best, "unit": "cell-updates/s",
            "h2d_bytes_per_step": h2d / sc.steps, "d2h_bytes_per_step": d2h / sc.steps,
            "h2d_bytes_per_run": h2d, "d2h_bytes_per_run": d2h,
            "run": f"one {sc.steps}-step run of {sc.name} through the C ABI: H2D of the initial "
                   f"state from pinned memory, {sc.steps} automaton steps, D2H of the final grid "
                   f"+ counters; per-step bytes are the run's bytes / {sc.steps}",
            "l2": "a single instance: its state stays in the L2 across the run's steps (the "
                  "simulation's own regime), unlike the headline's four instances in turn",
            "seconds_per_run": best, "final_moved": st["moved"]}


def large_inputs_leg(P, torch, sc, stream, instances=4, steps=96):
    """The headline scenario with inputs larger than L2 instead of a flush:
    `instances` independent copies (seeds sc.seed + k; 4 x 105 MiB > 129 MB
    L2) advanced together as a batch, so every step streams its planes from
    HBM; graph replays timed with one event pair (no per-step events)."""
    scs = [sc.with_(seed=sc.seed + k, name=f"{sc.name}#{k}") for k in range(instances)]
    b = P.Batch(scs, stream=stream)
    b.step(32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) * 1e-3 / steps  # per batched step
    status = b.device_status()
    b.close()
    algo = ALGO_BYTES_PER_CELL[sc.model] * sc.cells * instances
    peak, kind = measured_peak()
    return {"instances": instances, "steps": steps, "bytes_per_step": algo,
            "us_per_scenario_step": dt * 1e6 / instances,
            "cell_updates_per_s": sc.cells * instances / dt, "algorithmic_GBps": algo / dt / 1e9,
            "frac_of_peak": algo / dt / 1e9 / peak, "peak_kind": kind, "device_status": status}


def probe_leg(P, torch, stream, steps=20):
    """The 8192^2 probe at the same density (1.6M agents): 1.2 GB of planes
    per step, far beyond the 129 MB L2, so every step streams from HBM."""
    sc = WL.ACO_8192
    sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
    sim.place(sc.seed)
    sim.step(16)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) * 1e-3 / steps
    status = sim.device_status()
    sim.close()
    algo = ALGO_BYTES_PER_CELL[sc.model] * sc.cells
    peak, kind = measured_peak()
    return {"workload": sc.name, "steps": steps, "us_per_step": dt * 1e6,
            "cell_updates_per_s": sc.cells / dt, "algorithmic_GBps": algo / dt / 1e9,
            "frac_of_peak": algo / dt / 1e9 / peak, "peak_kind": kind, "device_status": status}


def batched_leg(P, torch, stream, count=256, steps=500):
    """The 256-scenario batch: autotuned launch configuration, then `steps`
    steps in batched launches, against the same scenarios and steps run one
    scenario at a time (each scenario's own launches, back to back on the
    same stream)."""
    from paper_1412_4933_gb300 import autotune
    scs = WL.batched_scenarios(count=count, steps=steps)
    cells = sum(s.cells for s in scs)
    algo = sum(ALGO_BYTES_PER_CELL[s.model] * s.cells for s in scs)  # bytes per batched step
    choice = autotune.tune(scs, stream=stream)
    batch = P.Batch(scs, stream=stream)
    autotune.apply(batch, choice)
    batch.step(16)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    status = batch.device_status()
    batch.close()
    # the same scenarios and steps, one scenario at a time
    sims = []
    for sc in scs:
        sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
        sim.set_variant(choice[0])
        if choice[0] not in (P.VARIANT_AGENT, P.VARIANT_DEFERRED):
            sim.set_tiling(choice[1], choice[2], choice[3])
        sim.place(sc.seed)
        sim.step(16)
        sims.append(sim)
    torch.cuda.synchronize()
    e0.record(stream)
    for sim in sims:
        sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) * 1e-3
    for sim in sims:
        sim.close()
    peak, kind = measured_peak()
    cpu = oracle_multicore(scs, steps=50, cores=min(16, os.cpu_count() or 1))
    return {"scenarios": count, "steps": steps, "cells": cells,
            "cpu_oracle_multicore": cpu,
            "launch_config": {"variant": choice[0], "tile": [choice[1], choice[2]],
                              "ctas_per_sm": choice[3]},
            "scenarios_per_s": count / t_batch,
            "cell_updates_per_s": cells * steps / t_batch,
            "algorithmic_bytes_per_step": algo,
            "algorithmic_bytes_note": "every-step evaporation: 18 B per ACO cell, 2 B per LEM "
                                      "cell (the deferred variant moves 18/32 B per ACO cell of "
                                      "dense traffic plus the agents' sparse accesses)",
            "algorithmic_GBps": algo * steps / t_batch / 1e9,
            "algorithmic_frac_of_peak": algo * steps / t_batch / 1e9 / peak, "peak_kind": kind,
            "one_scenario_at_a_time_cell_updates_per_s": cells * steps / t_single,
            "one_scenario_at_a_time": f"the same {count} scenarios x {steps} steps, each "
                                      f"scenario's own launches (same variant), back to back",
            "speedup_vs_one_scenario_at_a_time": t_single / t_batch,
            "device_status": status}


DEFER_PERIOD = 32  # the library's rolling-refresh period of the deferred step


def deferred_leg(P, torch, sc, stream, warmup: int, steps: int, repeats: int, headline_s: float):
    """The <18 B per cell-step scheme: the same step with deferred
    evaporation (per-cell stamps, values brought up to date where read and
    in a rolling refresh of 1/32 of the cells per step; bit-identical
    results), timed exactly like the headline: four instances in turn, one
    graph of `steps` steps, median of `repeats` replays."""
    sims = rotating_instances(P, torch, sc, stream, P.VARIANT_DEFERRED, warmup, ROTATING_INSTANCES)
    g = capture_steps(sims, torch, stream, steps)
    region = time_graph_repeats(g, torch, stream, repeats)
    del g
    status = max(abs(x.device_status()) for x in sims)
    for x in sims:
        x.close()
    step_s = statistics.median(region) / steps
    dense = 18.0 / DEFER_PERIOD if sc.model == WL.ACO else 0.0
    return {"variant": "deferred", "steps": steps, "repeats": len(region),
            "us_per_step": step_s * 1e6,
            "us_per_step_regions": [r * 1e6 / steps for r in region],
            "cell_updates_per_s": sc.cells / step_s,
            "speedup_vs_headline_step": headline_s / step_s,
            "dense_bytes_per_cell_step": dense,
            "dense_bytes_per_step": dense * sc.cells,
            "note": "one pass over every cell every 32 steps (18 B/cell) instead of every step; "
                    "the agents' accesses (positions, 3x3 occupancy, pheromone and stamps of "
                    "blocked agents, code planes, winners' writes) come on top and dominate",
            "gpu_launches_per_step": 2,
            "device_status": status}


def domain_leg(P, torch, sc, stream, warmup: int, steps: int, headline_s: float, n_strips=2):
    """The headline workload advanced as `n_strips` column strips on this one
    GPU (``sim_step_strip`` per strip; before every step each strip's three
    halo columns are refreshed from its neighbours' interiors), from the
    state a placed scenario reaches after `warmup` steps.  Here the halo
    exchange is one ``sim_strip_halo`` kernel per halo between the strips'
    tensors on one device; between GPUs it is point-to-point sends
    (domain.DistExchange), which one GPU cannot time."""
    from paper_1412_4933_gb300 import domain as D
    sim = P.Sim(sc.W, sc.H, P.params_of(sc), stream=stream)
    with torch.cuda.stream(stream):
        sim.place(sc.seed)
        sim.step(warmup)
    grid, agents = sim.read_grid(), sim.read_agents()
    sim.close()
    dom = D.StripDomain(sc.W, sc.H, P.params_of(sc), sc.seed, n_strips)
    with torch.cuda.stream(stream):
        dom.load(warmup, grid, agents)
        dom.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dom.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
    step_s = e0.elapsed_time(e1) * 1e-3 / steps
    return {"strips": n_strips, "steps": steps, "us_per_step": step_s * 1e6,
            "cell_updates_per_s": sc.cells / step_s,
            "single_grid_us_per_step": headline_s * 1e6,
            "exchange": "one sim_strip_halo kernel per halo between the strips' tensors "
                        "on one GPU; per step two halo copies and two sim_step_strip calls "
                        "issued from Python"}


def serving_leg(P, torch, stream, n_requests=200, budget_frac=0.5, chunk=16, warmup=4):
    """Poisson request stream (200/s) through the continuous-batching loop,
    after `warmup` requests of another stream served untimed on the same
    loop (the pool's memory and graphs exist before the timed stream)."""
    from paper_1412_4933_gb300 import serving
    reqs = WL.serving_requests(n_requests)
    free, _ = torch.cuda.mem_get_info()
    loop = serving.ServingLoop(int(free * budget_frac), 512, chunk=chunk, stream=stream)
    loop.run(WL.serving_requests(warmup, arrival_seed=8), realtime=False)
    rep = loop.run(reqs)
    loop.close()
    out = rep.summary()
    out.update({"rate_per_s": 200.0, "hbm_budget_frac": budget_frac, "chunk_steps": chunk,
                "warmup_requests": warmup})
    return out


def run_gpu(args, sc):
    import torch
    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1412_4933_gb300 import pedsim as P

    stream = torch.cuda.Stream(device)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    clean_buf = torch.ones(L2_FLUSH_BYTES // 8, dtype=torch.float32, device=device)

    def flush():
        # write a buffer larger than L2, then read another one so that the
        # dirty lines of the write are written back before the step starts
        with torch.cuda.stream(stream):
            flush_buf.fill_(1.0)
            clean_buf.sum()

    def flush_write_only():
        with torch.cuda.stream(stream):
            flush_buf.fill_(1.0)

    variant = VARIANTS[args.variant](P)
    # inputs larger than L2: ROTATING_INSTANCES resident copies of the
    # workload, stepped in turn, so that every step reads its state from HBM
    sims = rotating_instances(P, torch, sc, stream, variant, args.warmup, ROTATING_INSTANCES)
    sim = sims[0]
    graph = capture_steps(sims, torch, stream, args.steps)
    barrier(dist, device)

    with ClockSampler(local) as clk:
        region_s = time_graph_repeats(graph, torch, stream, args.repeats, dist, device)
    elapsed_max = statistics.median(region_s)
    clocks = clk.summary()
    status = max(abs(x.device_status()) for x in sims)
    launches = sim.launches_per_step()
    del graph
    for x in sims[1:]:
        x.close()
    # the same single-scenario step with the L2 flushed before each step and
    # an event pair around each step
    per_step = time_steps_flushed(sim, torch, stream, args.steps, flush)
    fl_s = sum(per_step) / len(per_step)

    cells_total = sc.cells * args.steps * world
    value = cells_total / elapsed_max
    ms_per_step = elapsed_max * 1e3 / args.steps

    # roofline of the step: algorithmic bytes / time.  The per-step time holds
    # both of the step's kernels (the first streams the bytes with the
    # proposals interleaved, the resolution follows it), so this is a lower
    # bound of the streaming part's rate
    algo_bytes = ALGO_BYTES_PER_CELL[sc.model] * sc.cells
    peak, peak_kind = measured_peak()
    step_s = elapsed_max / args.steps
    achieved = algo_bytes / step_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac_of_nominal": achieved / NOMINAL_HBM_GBPS, "nominal_peak": NOMINAL_HBM_GBPS,
                "frac": achieved / peak,
                "traffic": recorded_traffic() if args.variant == "agent" else None,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes,
                "kernel": KERNEL_NAMES[args.variant]}

    extra = {"flushed_per_step": {
        "steps": len(per_step), "us_per_step": fl_s * 1e6, "cell_updates_per_s": sc.cells / fl_s,
        "algorithmic_GBps": algo_bytes / fl_s / 1e9, "frac_of_peak": algo_bytes / fl_s / 1e9 / peak,
        "l2": "flushed before each step (512 MB write, then a 256 MB read of another buffer), "
              "one event pair per step"}}
    if rank == 0 and not args.quick:
        # the same steps with the write-only flush (its write-backs land in
        # the step)
        wo = time_steps_flushed(sim, torch, stream, min(args.steps, 100), flush_write_only)
        wo_s = sum(wo) / len(wo)
        extra["flushed_write_only"] = {"steps": len(wo), "us_per_step": wo_s * 1e6,
                                       "cell_updates_per_s": sc.cells / wo_s,
                                       "algorithmic_GBps": algo_bytes / wo_s / 1e9}
        # steady state: back-to-back steps (graph replays), no flush
        with torch.cuda.stream(stream):
            sim.step(32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steady_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st_s = e0.elapsed_time(e1) * 1e-3
        extra["steady"] = {"steps": args.steady_steps, "cell_updates_per_s": sc.cells * args.steady_steps / st_s,
                           "us_per_step": st_s * 1e6 / args.steady_steps,
                           "algorithmic_GBps": algo_bytes * args.steady_steps / st_s / 1e9,
                           "l2": "resident (no flush)"}
    sim.close()

    e2e = None
    if rank == 0 and not args.quick:
        e2e = e2e_run(P, torch, sc, stream, reps=2)
    if rank == 0 and args.variant == "agent":
        extra["deferred_evaporation"] = deferred_leg(P, torch, sc, stream, args.warmup, args.steps,
                                                     args.repeats, elapsed_max / args.steps)
    if rank == 0 and not args.quick and not args.no_probe:
        extra["hbm_probe"] = probe_leg(P, torch, stream)
        extra["inputs_larger_than_l2"] = large_inputs_leg(P, torch, sc, stream)
    if rank == 0 and not args.quick and not args.no_batched:
        extra["batched"] = batched_leg(P, torch, stream)
    if rank == 0 and not args.quick and not args.no_domain:
        extra["domain_strips"] = domain_leg(P, torch, sc, stream, args.warmup, args.steps,
                                            elapsed_max / args.steps)
    if rank == 0 and not args.quick and not args.no_serving:
        extra["serving"] = serving_leg(P, torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        cpu_steps = args.cpu_steps
        rate, dt = oracle_rate(sc, cpu_steps)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"first {cpu_steps} steps of {sc.name} after placement "
                         f"({dt:.1f} s, single-threaded)",
               "host_cores_available": os.cpu_count()}

    if rank == 0:
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sc.name, "W": sc.W, "H": sc.H, "agents": sc.agents,
                       "model": "ACO" if sc.model else "LEM", "rho": sc.rho, "seed": sc.seed,
                       "band_cols": sc.band_cols,
                       "l2": rotating_l2_note(P, sc),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "timed_regions": {
                "repeats": len(region_s), "steps_each": args.steps,
                "us_per_step": [r * 1e6 / args.steps for r in region_s],
                "median_us_per_step": elapsed_max * 1e6 / args.steps,
                "spread_us_per_step": (max(region_s) - min(region_s)) * 1e6 / args.steps,
                "note": "each region is one replay of one CUDA graph of exactly `steps` steps "
                        "(instances in turn), after one untimed replay; value and ms_per_step "
                        "are the median region"},
            "clocks": clocks, "gpu_launches": launches * args.steps,
            "device_status": status,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=HEADLINE_REPEATS,
                    help="timed regions of exactly --steps steps; the headline is their median")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WL.ACO_2048.name, choices=sorted(WL.SINGLE))
    ap.add_argument("--variant", default="agent", choices=sorted(VARIANTS),
                    help="step variant of the headline simulation")
    ap.add_argument("--steady-steps", type=int, default=2000)
    ap.add_argument("--cpu-steps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-domain", action="store_true",
                    help="skip the column-strip decomposition leg")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline only (for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.repeats < 1 or args.steps < 1:
        ap.error("--repeats and --steps must be >= 1")
    sc = WL.SINGLE[args.workload]
    if args.impl == "reference":
        return run_reference(args, sc)
    return run_gpu(args, sc)


if __name__ == "__main__":
    sys.exit(main())
