"""Thin Python binding of the C ABI in ``include/pedsim.h`` (ctypes).

Argument marshalling only: every step of the automaton runs in the CUDA
kernels of ``libpedsim.so``.  Importing this module loads that library and
raises ``ImportError`` when it has not been built (``__graft_entry__.build()``
or ``python -m paper_1412_4933_gb300.build``); there is no CPU fallback.

Streams: by default each handle runs on PyTorch's current CUDA stream when
PyTorch is importable and a GPU is present, else on the legacy default stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpedsim.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first (paper_1412_4933_gb300.build.build())")

_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ENOSPC, ECUDA, ETIMEDOUT, ENOENT = 0, -22, -12, -28, -5, -110, -2
LEM, ACO = 0, 1
VARIANT_TILED, VARIANT_TWO_PASS, VARIANT_FUSED, VARIANT_AGENT, VARIANT_DEFERRED = 0, 1, 2, 3, 4
TEST_SKIP_RESOLVE_LOADS = 1


class SimParams(C.Structure):
    _fields_ = [("model", C.c_uint32), ("n_per_side", C.c_uint32), ("band_cols", C.c_uint32),
                ("rho", C.c_float), ("tau0", C.c_float), ("deposit", C.c_float),
                ("alpha", C.c_uint32), ("beta", C.c_uint32), ("deposit_mode", C.c_uint32),
                ("lem_sigma", C.c_float)]


class SimStats(C.Structure):
    _fields_ = [("step", C.c_uint64), ("agents", C.c_uint32 * 2), ("crossed", C.c_uint32 * 2),
                ("parked", C.c_uint32 * 2), ("moved", C.c_uint64), ("conflicts", C.c_uint64)]

    def as_dict(self) -> dict:
        return {"step": int(self.step), "agents": list(self.agents),
                "crossed": list(self.crossed), "parked": list(self.parked),
                "moved": int(self.moved), "conflicts": int(self.conflicts)}


_P = C.c_void_p
_SIGS = {
    "sim_default_params": (None, [C.POINTER(SimParams)]),
    "sim_validate": (C.c_int, [C.c_int, C.c_int, C.POINTER(SimParams)]),
    "sim_device_bytes": (C.c_size_t, [C.c_int, C.c_int, C.POINTER(SimParams)]),
    "sim_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(SimParams), C.POINTER(_P)]),
    "sim_set_stream": (C.c_int, [_P, _P]),
    "sim_place": (C.c_int, [_P, C.c_uint64]),
    "sim_step": (C.c_int, [_P, C.c_int]),
    "sim_read_grid": (C.c_int, [_P, _P, _P, _P, _P]),
    "sim_read_agents": (C.c_int, [_P, _P, _P]),
    "sim_set_state": (C.c_int, [_P, C.c_uint64, C.c_uint64, _P, _P, _P, _P, _P, _P]),
    "sim_stats": (C.c_int, [_P, C.POINTER(SimStats)]),
    "sim_save": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "sim_load": (C.c_int, [_P, _P, C.c_size_t]),
    "sim_set_variant": (C.c_int, [_P, C.c_int]),
    "sim_set_tiling": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "sim_device_status": (C.c_int, [_P]),
    "sim_set_wait_test": (C.c_int, [_P, C.c_uint64, C.c_uint32]),
    "sim_launches_per_step": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "sim_destroy": (None, [_P]),
    "sim_last_error": (C.c_char_p, [_P]),
    "sim_batch_create": (C.c_int, [C.c_int, _P, _P, _P, _P, C.POINTER(_P)]),
    "sim_batch_set_stream": (C.c_int, [_P, _P]),
    "sim_batch_step": (C.c_int, [_P, C.c_int]),
    "sim_batch_stats": (C.c_int, [_P, C.c_int, C.POINTER(SimStats)]),
    "sim_batch_read_grid": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "sim_batch_set_variant": (C.c_int, [_P, C.c_int]),
    "sim_batch_set_tiling": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "sim_batch_device_status": (C.c_int, [_P]),
    "sim_batch_destroy": (None, [_P]),
    "sim_batch_last_error": (C.c_char_p, [_P]),
    "sim_pool_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_P)]),
    "sim_pool_set_stream": (C.c_int, [_P, _P]),
    "sim_pool_admit": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(SimParams), C.c_uint64,
                                 C.c_uint64, C.POINTER(C.c_int)]),
    "sim_pool_step": (C.c_int, [_P, C.c_int]),
    "sim_pool_finished": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int)]),
    "sim_pool_stats": (C.c_int, [_P, C.c_int, C.POINTER(SimStats)]),
    "sim_pool_read_grid": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "sim_pool_release": (C.c_int, [_P, C.c_int]),
    "sim_pool_bytes_in_use": (C.c_size_t, [_P]),
    "sim_pool_live": (C.c_int, [_P]),
    "sim_pool_destroy": (None, [_P]),
    "sim_pool_last_error": (C.c_char_p, [_P]),
    "sim_step_noalloc": (C.c_int, [C.c_int, C.c_int, C.POINTER(SimParams), C.c_uint64, C.c_uint64,
                                   _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sim_step_strip": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(SimParams), C.c_uint64, C.c_uint64,
                                 _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sim_strip_halo": (C.c_int, [C.c_int, C.c_int, C.c_uint32, _P, _P, _P, _P, _P, _P,
                                 C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, C.c_int, C.c_int, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class PedsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pedsim error {code}: {msg}")
        self.code = code


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def make_params(model=LEM, n_per_side=0, band_cols=16, rho=0.05, tau0=1.0, deposit=1.0,
                alpha=1, beta=1, deposit_mode=0, lem_sigma=1.0) -> SimParams:
    return SimParams(model, n_per_side, band_cols, rho, tau0, deposit, alpha, beta,
                     deposit_mode, lem_sigma)


def params_of(scenario) -> SimParams:
    """SimParams of a ``workloads.Scenario``."""
    return make_params(**scenario.params())


def device_bytes(W: int, H: int, params: SimParams) -> int:
    return int(_lib.sim_device_bytes(W, H, C.byref(params)))


def validate(W: int, H: int, params: SimParams) -> int:
    return int(_lib.sim_validate(W, H, C.byref(params)))


class Sim:
    """One scenario on the GPU (``sim_create`` ... ``sim_destroy``)."""

    def __init__(self, W: int, H: int, params: SimParams, stream=None):
        h = _P()
        rc = _lib.sim_create(W, H, C.byref(params), C.byref(h))
        if rc != 0:
            raise PedsimError(rc, "sim_create rejected the scenario")
        self._h = h
        self.W, self.H, self.params = W, H, params
        self.n_agents = 2 * params.n_per_side
        self.set_stream(stream if stream is not None else _default_stream())

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise PedsimError(rc, (_lib.sim_last_error(self._h) or b"").decode())

    def set_stream(self, stream) -> None:
        if stream is not None and not isinstance(stream, C.c_void_p):
            stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._check(_lib.sim_set_stream(self._h, stream))

    def place(self, seed: int) -> None:
        self._check(_lib.sim_place(self._h, seed))

    def step(self, n: int = 1) -> None:
        self._check(_lib.sim_step(self._h, n))

    def set_variant(self, variant: int) -> None:
        self._check(_lib.sim_set_variant(self._h, variant))

    def set_tiling(self, tile_w: int, tile_h: int, ctas_per_sm: int = 0) -> None:
        self._check(_lib.sim_set_tiling(self._h, tile_w, tile_h, ctas_per_sm))

    def read_grid(self, occ=True, ids=True, tau=True) -> dict:
        cells = self.W * self.H
        o = np.empty(cells, np.uint8) if occ else None
        i = np.empty(cells, np.uint32) if ids else None
        a = np.empty(cells, np.float32) if tau else None
        b = np.empty(cells, np.float32) if tau else None
        self._check(_lib.sim_read_grid(self._h, _ptr(o), _ptr(i), _ptr(a), _ptr(b)))
        shp = (self.H, self.W)
        out = {}
        if occ: out["occ"] = o.reshape(shp)
        if ids: out["ids"] = i.reshape(shp)
        if tau:
            out["tauA"] = a.reshape(shp)
            out["tauB"] = b.reshape(shp)
        return out

    def read_agents(self) -> dict:
        n = self.n_agents + 1
        arr = np.empty(n, np.uint32)
        tour = np.empty(n, np.float32)
        self._check(_lib.sim_read_agents(self._h, _ptr(arr), _ptr(tour)))
        return {"arrival": arr, "tour": tour}

    def set_state(self, seed: int, step: int, occ, ids, tauA=None, tauB=None, arrival=None,
                  tour=None) -> None:
        conv = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt).reshape(-1)
        occ, ids = conv(occ, np.uint8), conv(ids, np.uint32)
        tauA, tauB = conv(tauA, np.float32), conv(tauB, np.float32)
        arrival, tour = conv(arrival, np.uint32), conv(tour, np.float32)
        self._check(_lib.sim_set_state(self._h, seed, step, _ptr(occ), _ptr(ids), _ptr(tauA),
                                       _ptr(tauB), _ptr(arrival), _ptr(tour)))

    def stats(self) -> dict:
        st = SimStats()
        self._check(_lib.sim_stats(self._h, C.byref(st)))
        return st.as_dict()

    def save(self) -> bytes:
        n = C.c_size_t(0)
        self._check(_lib.sim_save(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(_lib.sim_save(self._h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes) -> None:
        buf = C.create_string_buffer(blob, len(blob))
        self._check(_lib.sim_load(self._h, buf, len(blob)))

    def device_status(self) -> int:
        return int(_lib.sim_device_status(self._h))

    def set_wait_test(self, wait_cycles: int = 0, flags: int = 0) -> None:
        """Failure-detection test hook (``sim_set_wait_test``)."""
        self._check(_lib.sim_set_wait_test(self._h, wait_cycles, flags))

    def launches_per_step(self) -> int:
        """Kernel launches of one step(1) call with the current variant."""
        n = C.c_int(0)
        self._check(_lib.sim_launches_per_step(self._h, C.byref(n)))
        return int(n.value)

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h:
            _lib.sim_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h


class Batch:
    """Many independent scenarios stepped together (``sim_batch_*``)."""

    def __init__(self, scenarios, stream=None):
        n = len(scenarios)
        Ws = np.array([s.W for s in scenarios], np.int32)
        Hs = np.array([s.H for s in scenarios], np.int32)
        prm = (SimParams * n)(*[params_of(s) for s in scenarios])
        seeds = np.array([s.seed for s in scenarios], np.uint64)
        self.scenarios = list(scenarios)
        h = _P()
        # placement runs on the default stream before the handle's own stream is set
        rc = _lib.sim_batch_create(n, _ptr(Ws), _ptr(Hs), C.cast(prm, C.c_void_p), _ptr(seeds),
                                   C.byref(h))
        if rc != 0:
            raise PedsimError(rc, "sim_batch_create failed")
        self._h = h
        st = stream if stream is not None else _default_stream()
        if st is not None and not isinstance(st, C.c_void_p):
            st = C.c_void_p(int(getattr(st, "cuda_stream", st)))
        self._check(_lib.sim_batch_set_stream(self._h, st))

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise PedsimError(rc, (_lib.sim_batch_last_error(self._h) or b"").decode())

    def step(self, n: int = 1) -> None:
        self._check(_lib.sim_batch_step(self._h, n))

    def set_variant(self, variant: int) -> None:
        self._check(_lib.sim_batch_set_variant(self._h, variant))

    def set_tiling(self, tile_w: int, tile_h: int, ctas_per_sm: int = 0) -> None:
        self._check(_lib.sim_batch_set_tiling(self._h, tile_w, tile_h, ctas_per_sm))

    def stats(self, i: int) -> dict:
        st = SimStats()
        self._check(_lib.sim_batch_stats(self._h, i, C.byref(st)))
        return st.as_dict()

    def read_grid(self, i: int) -> dict:
        sc = self.scenarios[i]
        cells = sc.W * sc.H
        o, ids = np.empty(cells, np.uint8), np.empty(cells, np.uint32)
        a, b = np.empty(cells, np.float32), np.empty(cells, np.float32)
        self._check(_lib.sim_batch_read_grid(self._h, i, _ptr(o), _ptr(ids), _ptr(a), _ptr(b)))
        shp = (sc.H, sc.W)
        return {"occ": o.reshape(shp), "ids": ids.reshape(shp), "tauA": a.reshape(shp),
                "tauB": b.reshape(shp)}

    def device_status(self) -> int:
        return int(_lib.sim_batch_device_status(self._h))

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h:
            _lib.sim_batch_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class Pool:
    """Serving pool of device-resident scenario slots (``sim_pool_*``)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, stream=None):
        h = _P()
        rc = _lib.sim_pool_create(hbm_budget_bytes, max_slots, C.byref(h))
        if rc != 0:
            raise PedsimError(rc, "sim_pool_create failed")
        self._h = h
        self.max_slots = max_slots
        st = stream if stream is not None else _default_stream()
        if st is not None and not isinstance(st, C.c_void_p):
            st = C.c_void_p(int(getattr(st, "cuda_stream", st)))
        self._check(_lib.sim_pool_set_stream(self._h, st))

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise PedsimError(rc, (_lib.sim_pool_last_error(self._h) or b"").decode())

    def admit(self, scenario, steps=None):
        """Slot id, or None when the HBM budget / slot count is exhausted."""
        slot = C.c_int(-1)
        p = params_of(scenario)
        rc = _lib.sim_pool_admit(self._h, scenario.W, scenario.H, C.byref(p), scenario.seed,
                                 scenario.steps if steps is None else steps, C.byref(slot))
        if rc == ENOSPC:
            return None
        self._check(rc)
        return slot.value

    def step(self, n: int) -> None:
        self._check(_lib.sim_pool_step(self._h, n))

    def finished(self) -> list:
        buf = np.empty(self.max_slots, np.int32)
        n = C.c_int(0)
        self._check(_lib.sim_pool_finished(self._h, _ptr(buf), self.max_slots, C.byref(n)))
        return [int(v) for v in buf[: n.value]]

    def stats(self, slot: int) -> dict:
        st = SimStats()
        self._check(_lib.sim_pool_stats(self._h, slot, C.byref(st)))
        return st.as_dict()

    def read_grid(self, slot: int, W: int, H: int) -> dict:
        cells = W * H
        o, ids = np.empty(cells, np.uint8), np.empty(cells, np.uint32)
        a, b = np.empty(cells, np.float32), np.empty(cells, np.float32)
        self._check(_lib.sim_pool_read_grid(self._h, slot, _ptr(o), _ptr(ids), _ptr(a), _ptr(b)))
        return {"occ": o.reshape(H, W), "ids": ids.reshape(H, W), "tauA": a.reshape(H, W),
                "tauB": b.reshape(H, W)}

    def release(self, slot: int) -> None:
        self._check(_lib.sim_pool_release(self._h, slot))

    @property
    def bytes_in_use(self) -> int:
        return int(_lib.sim_pool_bytes_in_use(self._h))

    @property
    def live(self) -> int:
        return int(_lib.sim_pool_live(self._h))

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h:
            _lib.sim_pool_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


NOALLOC_MAX_CELLS = 1 << 24


def step_noalloc(W, H, params: SimParams, seed: int, step: int, occ_in, occ_out, ids, tauA_in=None,
                 tauB_in=None, tauA_out=None, tauB_out=None, arrival=None, tour=None,
                 counters=None, stream=None) -> int:
    """One allocation-free step on caller-owned device tensors (anything with
    ``data_ptr()``); returns the C status code.  For callers that must not let
    the library allocate device memory: the scratch it needs lives in a fixed
    device array of the library (at most NOALLOC_MAX_CELLS cells)."""
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    if stream is None:
        stream = _default_stream()
    elif not isinstance(stream, C.c_void_p):
        stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    return int(_lib.sim_step_noalloc(W, H, C.byref(params), seed, step, ptr(occ_in), ptr(occ_out),
                                     ptr(ids), ptr(tauA_in), ptr(tauB_in), ptr(tauA_out),
                                     ptr(tauB_out), ptr(arrival), ptr(tour), ptr(counters), stream))


def step_strip(W, H, x0, W_global, interior_lo, interior_hi, params: SimParams, seed: int,
               step: int, occ_in, occ_out, ids, tauA_in, tauB_in, tauA_out, tauB_out, arrival,
               tour, scratch, counters=None, stream=None) -> int:
    """One step of a column strip of a W_global x H grid on caller-owned
    device tensors (``sim_step_strip``); returns the C status code."""
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    if stream is None:
        stream = _default_stream()
    elif not isinstance(stream, C.c_void_p):
        stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    return int(_lib.sim_step_strip(W, H, x0, W_global, interior_lo, interior_hi, C.byref(params),
                                   seed, step, ptr(occ_in), ptr(occ_out), ptr(ids), ptr(tauA_in),
                                   ptr(tauB_in), ptr(tauA_out), ptr(tauB_out), ptr(arrival),
                                   ptr(tour), ptr(scratch), ptr(counters), stream))


def strip_halo(H, ncols, n_agents, src, src_W, src_col, dst, dst_W, dst_col,
               stream=None) -> int:
    """Halo copy between two strips on one device (``sim_strip_halo``):
    `src` and `dst` are (occ, ids, tauA, tauB, arrival, tour) device
    tensors (tauA/tauB None for LEM, tour None when neither keeps one);
    returns the C status code."""
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    if stream is None:
        stream = _default_stream()
    elif not isinstance(stream, C.c_void_p):
        stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    return int(_lib.sim_strip_halo(H, ncols, n_agents, *(ptr(t) for t in src), src_W, src_col,
                                   *(ptr(t) for t in dst), dst_W, dst_col, stream))


def exported_symbols():
    """Names of the C-ABI functions this binding declares."""
    return sorted(_SIGS)
