"""ctypes wrapper around the C oracle (``pedsim_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports
this module.

The oracle is the paper's per-step update written out literally (Sec. III-IV
of Dutta, McLeod, Friesen): agents decide a FUTURE cell (Sec. IV.b-c, Eq. 1,
Eq. 2), then empty cells gather their claimants and pick one (Sec. IV.d),
pheromone evaporates (Eq. 3) and is deposited (Eq. 4, Eq. 5).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pedsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Flags: plain IEEE binary32 with no contraction into FMA and no fast-math,
# so that the float operations happen exactly in the written order.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, a second or two)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


class Params(C.Structure):
    """Mirror of ``orc_params`` in the C oracle."""
    _fields_ = [("model", C.c_uint32), ("n_per_side", C.c_uint32),
                ("band_cols", C.c_uint32), ("rho", C.c_float), ("tau0", C.c_float),
                ("deposit", C.c_float), ("alpha", C.c_uint32), ("beta", C.c_uint32),
                ("deposit_mode", C.c_uint32), ("lem_sigma", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_uint64), ("agents", C.c_uint32 * 2),
                ("crossed", C.c_uint32 * 2), ("parked", C.c_uint32 * 2),
                ("moved", C.c_uint64), ("conflicts", C.c_uint64)]

    def as_dict(self) -> dict:
        return {"step": int(self.step), "agents": list(self.agents),
                "crossed": list(self.crossed), "parked": list(self.parked),
                "moved": int(self.moved), "conflicts": int(self.conflicts)}


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.orc_philox4x64_10.argtypes = [C.POINTER(C.c_uint64)] * 3
        L.orc_eta.argtypes = [C.c_int]; L.orc_eta.restype = C.c_float
        L.orc_lem_rank.argtypes = [C.c_int32, C.c_int, C.c_float]; L.orc_lem_rank.restype = C.c_int
        L.orc_lem_rank_table.argtypes = [C.c_int, C.c_float, C.c_void_p]
        L.orc_aco_weight.argtypes = [C.c_float, C.c_float, C.c_uint32, C.c_uint32]
        L.orc_aco_weight.restype = C.c_float
        L.orc_aco_pick.argtypes = [C.POINTER(C.c_float), C.c_uint32]; L.orc_aco_pick.restype = C.c_int
        L.orc_aco_histogram.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_uint64)]
        L.orc_conflict_index.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_conflict_index.restype = C.c_uint32
        L.orc_check_params.argtypes = [C.c_int, C.c_int, C.POINTER(Params)]
        L.orc_check_params.restype = C.c_int
        L.orc_create.argtypes = [C.c_int, C.c_int, C.POINTER(Params), C.c_uint64, C.c_int]
        L.orc_create.restype = P
        L.orc_create_from_state.argtypes = [C.c_int, C.c_int, C.POINTER(Params), C.c_uint64,
                                            C.c_uint64, C.c_int, P, P, P, P, P]
        L.orc_create_from_state.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_step.argtypes = [P, C.c_int]; L.orc_step.restype = C.c_int
        L.orc_get_state.argtypes = [P, P, P, P, P, P, P]
        L.orc_get_stats.argtypes = [P, C.POINTER(Stats)]
        L.orc_decide_at.argtypes = [P, C.c_int, C.c_int]; L.orc_decide_at.restype = C.c_int
        L.orc_n_agents.argtypes = [P]; L.orc_n_agents.restype = C.c_uint32
        L.orc_current_step.argtypes = [P]; L.orc_current_step.restype = C.c_uint64
        _lib = L
    return _lib


def make_params(model=0, n_per_side=0, band_cols=16, rho=0.05, tau0=1.0, deposit=1.0,
                alpha=1, beta=1, deposit_mode=0, lem_sigma=1.0) -> Params:
    return Params(model, n_per_side, band_cols, rho, tau0, deposit, alpha, beta,
                  deposit_mode, lem_sigma)


def philox4x64_10(ctr, key):
    """One Philox4x64-10 block: four 64-bit counter words, two key words."""
    c = (C.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One scenario advanced step by step on the CPU."""

    def __init__(self, W, H, params: Params, seed: int, mirror: bool = False, *,
                 state=None, step: int = 0):
        L = lib()
        self.W, self.H, self.params, self.seed = W, H, params, seed
        if state is None:
            h = L.orc_create(W, H, C.byref(params), seed, int(mirror))
        else:
            occ = np.ascontiguousarray(state["occ"], dtype=np.uint8).reshape(-1)
            ids = np.ascontiguousarray(state["ids"], dtype=np.uint32).reshape(-1)
            tA = state.get("tauA"); tB = state.get("tauB"); arr = state.get("arrival")
            tA = None if tA is None else np.ascontiguousarray(tA, dtype=np.float32).reshape(-1)
            tB = None if tB is None else np.ascontiguousarray(tB, dtype=np.float32).reshape(-1)
            arr = None if arr is None else np.ascontiguousarray(arr, dtype=np.uint32)
            h = L.orc_create_from_state(W, H, C.byref(params), seed, step, int(mirror),
                                        _ptr(occ), _ptr(ids), _ptr(tA), _ptr(tB), _ptr(arr))
        if not h:
            raise ValueError("oracle rejected the parameters or the state")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def n_agents(self) -> int:
        return int(lib().orc_n_agents(self._h))

    @property
    def step_index(self) -> int:
        return int(lib().orc_current_step(self._h))

    def step(self, n: int = 1) -> None:
        if lib().orc_step(self._h, n) != 0:
            raise ValueError("bad step count")

    def state(self) -> dict:
        cells = self.W * self.H
        occ = np.empty(cells, np.uint8); ids = np.empty(cells, np.uint32)
        tA = np.empty(cells, np.float32); tB = np.empty(cells, np.float32)
        arr = np.empty(self.n_agents + 1, np.uint32); tour = np.empty(self.n_agents + 1, np.float32)
        lib().orc_get_state(self._h, _ptr(occ), _ptr(ids), _ptr(tA), _ptr(tB), _ptr(arr), _ptr(tour))
        shp = (self.H, self.W)
        return {"occ": occ.reshape(shp), "ids": ids.reshape(shp), "tauA": tA.reshape(shp),
                "tauB": tB.reshape(shp), "arrival": arr, "tour": tour}

    def stats(self) -> dict:
        st = Stats()
        lib().orc_get_stats(self._h, C.byref(st))
        return st.as_dict()

    def decide_at(self, x: int, y: int) -> int:
        return int(lib().orc_decide_at(self._h, x, y))


def timed_run(W: int, H: int, params: dict, seed: int, steps: int):
    """Places a scenario and times `steps` oracle steps; returns
    (W * H * steps, seconds).  Module-level so that a spawned process pool
    can run it (benchmark use: the oracle on several host cores at once)."""
    orc = Oracle(W, H, make_params(**params), seed)
    import time
    t0 = time.perf_counter()
    orc.step(steps)
    return W * H * steps, time.perf_counter() - t0
