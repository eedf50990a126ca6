"""Autotuner of the batched step's launch configuration.

Knobs: the step variant (tiled two-kernel step with 128 x 8 or 128 x 16
tiles, the fused persistent kernel with one of its tile shapes, the
agent-parallel step or its deferred-evaporation form, which have no tiles)
and, for the persistent kernel, the
CTAs per SM (how many tiles, possibly of different scenarios, an SM works on
at once).  Each candidate is timed on a scratch
batch built from the same scenario descriptions (so the tuned batch's own
state is never advanced), and the winner is cached per (GPU name, size
class) in a JSON file.  Every candidate gives bit-identical results, so the
choice only affects speed.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import pedsim as P

CANDIDATES = [
    (P.VARIANT_DEFERRED, 0, 0, 0),
    (P.VARIANT_AGENT, 0, 0, 0),
    (P.VARIANT_TILED, 128, 8, 0),
    (P.VARIANT_TILED, 128, 16, 0),
    (P.VARIANT_FUSED, 64, 16, 0),
    (P.VARIANT_FUSED, 64, 8, 0),
    (P.VARIANT_FUSED, 128, 8, 0),
    (P.VARIANT_FUSED, 64, 16, 8),
]

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pedsim_gb300", "autotune.json")


def size_class(scenarios) -> str:
    cells = sum(s.cells for s in scenarios)
    aco = sum(1 for s in scenarios if s.model == 1)
    return (f"n{2 ** max(0, math.ceil(math.log2(len(scenarios))))}"
            f"_cells2^{max(0, round(math.log2(max(cells, 1))))}"
            f"_aco{round(4 * aco / max(len(scenarios), 1))}of4")


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:  # pragma: no cover - no torch / no GPU
        return "unknown"


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(CACHE + ".tmp", CACHE)
    except OSError:
        pass


def apply(batch, choice) -> None:
    variant, tw, th, cps = choice
    batch.set_variant(variant)
    if variant not in (P.VARIANT_AGENT, P.VARIANT_DEFERRED):
        batch.set_tiling(tw, th, cps)


def tune(scenarios, steps: int = 32, candidates=CANDIDATES, use_cache: bool = True,
         stream=None, repeats: int = 2) -> tuple:
    """Best (variant, tile_w, tile_h, ctas_per_sm) for this batch of scenarios:
    each candidate runs 16 warm-up steps (graph capture), then is timed over
    `steps` steps `repeats` times; the best of its repeats counts."""
    import torch
    key = f"{_gpu_name()}|{size_class(scenarios)}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["choice"])
    scratch = P.Batch(scenarios, stream=stream)
    timings = []
    try:
        for cand in candidates:
            apply(scratch, cand)
            scratch.step(16)  # warm-up (graph capture)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(repeats):
                t0 = time.perf_counter()
                scratch.step(steps)
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            timings.append((best, cand))
    finally:
        scratch.close()
    best = min(timings)[1]
    if use_cache:
        cache[key] = {"choice": list(best), "timings_s": [[t, list(c)] for t, c in timings]}
        _store_cache(cache)
    return best
