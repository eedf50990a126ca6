"""The C-ABI library loads and exports every function include/pedsim.h
declares; host-only entry points (defaults, validation, sizing) behave as
documented.  No CUDA compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pedsim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = re.findall(r"\b(sim_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1412_4933_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("sim_create", "sim_place", "sim_step", "sim_read_grid", "sim_stats",
                 "sim_save", "sim_load", "sim_destroy", "sim_last_error", "sim_batch_create",
                 "sim_batch_step", "sim_batch_stats", "sim_pool_admit", "sim_pool_step"):
        assert core in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = C.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1412_4933_gb300 import pedsim as P
    assert sorted(P.exported_symbols()) == declared_functions()


def test_host_only_entry_points(lib_path):
    from paper_1412_4933_gb300 import pedsim as P
    p = P.SimParams()
    P._lib.sim_default_params(C.byref(p))
    assert (p.model, p.band_cols, p.alpha, p.beta, p.deposit_mode) == (0, 16, 1, 1, 0)
    assert abs(p.rho - 0.05) < 1e-7 and p.tau0 == 1.0 and p.lem_sigma == 1.0
    good = P.make_params(model=P.ACO, n_per_side=100, band_cols=8, rho=0.02)
    assert P.validate(64, 64, good) == P.OK
    for W, H, prm in [(60, 64, good), (64, 0, good),
                      (64, 64, P.make_params(model=P.ACO, n_per_side=600, band_cols=8)),
                      (64, 64, P.make_params(model=P.ACO, n_per_side=10, band_cols=40)),
                      (64, 64, P.make_params(model=P.ACO, n_per_side=10, band_cols=8, rho=0.0)),
                      (64, 64, P.make_params(model=P.ACO, n_per_side=10, band_cols=8, beta=7)),
                      (64, 64, P.make_params(model=3)),
                      (64, 64, P.make_params(lem_sigma=0.0))]:
        assert P.validate(W, H, prm) == P.EINVAL
        assert P.device_bytes(W, H, prm) == 0
    # ACO 2048^2 with 100K agents: 2 occupancy planes, the proposal plane,
    # 2 code planes, ids, 4 pheromone planes, the deferred-evaporation stamps
    # (26 bytes per cell) plus per-agent arrays (arrival, position, code:
    # 0.9 MB), counter slots and the tile-activity block
    from paper_1412_4933_gb300 import workloads as WL
    prm = P.params_of(WL.ACO_2048)
    nbytes = P.device_bytes(2048, 2048, prm)
    cells = 2048 * 2048
    assert 26 * cells <= nbytes < 26 * cells + 2 * 2**20
    # LEM keeps no pheromone planes: 2 occupancy, proposal, 2 code planes and
    # ids (9 bytes per cell) plus small arrays
    lem = P.params_of(WL.LEM_256)
    assert 9 * 256 * 256 <= P.device_bytes(256, 256, lem) < 10 * 256 * 256


def test_oracle_and_library_share_no_source():
    """The CUDA sources never include or name the oracle and vice versa."""
    csrc = os.path.join(ROOT, "paper_1412_4933_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    pkg = os.path.join(ROOT, "paper_1412_4933_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in text and "from oracle" not in text, f
    otext = open(os.path.join(ROOT, "oracle", "pedsim_oracle.c")).read()
    assert "#include \"" not in otext


def test_division_by_width_multiplier():
    """The kernels divide cell indices (< 2^31) by the grid width W with a
    multiplier and a shift computed on the host (round-up method of
    Granlund and Montgomery): floor(c / W) = umulhi(c, mul) >> shr with
    l = ceil(log2 W), mul = floor(2^(31+l) / W) + 1, shr = l - 1.  Checked
    against integer division for every width class the library accepts
    (multiples of 16, powers of two and not) on edge and random indices."""
    import numpy as np
    rng = np.random.default_rng(3)
    widths = [16, 32, 48, 96, 144, 176, 480, 1008, 1024, 1424, 2048, 4080, 8192, 65536,
              65552, 1 << 20, (1 << 27) - 16, 1 << 27]
    for W in widths:
        l = int(W - 1).bit_length()
        mul = (1 << (31 + l)) // W + 1
        shr = l - 1
        assert mul < (1 << 32)
        k = np.arange(1, 4096, dtype=np.int64)
        near = np.arange(min(4 * W, 65536), dtype=np.int64)
        c = np.concatenate([rng.integers(0, 1 << 31, 200_000, dtype=np.int64), near,
                            (1 << 31) - 1 - near, k * W - 1, k * W,
                            ((1 << 31) // W - k) * W, ((1 << 31) // W - k) * W - 1]).astype(np.uint64)
        c = c[c < (1 << 31)]
        q = ((c * np.uint64(mul)) >> np.uint64(32)) >> np.uint64(shr)
        assert np.array_equal(q, c // np.uint64(W)), W


def test_strip_halo_rejects_bad_arguments_before_any_launch(lib_path):
    """sim_strip_halo validates its columns and pointers on the host: every
    call here fails before a kernel could start (the pointers are never
    dereferenced)."""
    from paper_1412_4933_gb300 import pedsim as P
    f = P._lib.sim_strip_halo
    v = C.c_void_p(256)  # stand-in device pointer, never touched
    none = None

    def call(H=8, ncols=3, src_W=10, src_col=7, dst_W=10, dst_col=0,
             src_tau=(v, v), dst_tau=(v, v), src_tour=v, dst_tour=v, src_occ=v):
        return f(H, ncols, 10, src_occ, v, src_tau[0], src_tau[1], v, src_tour, src_W, src_col,
                 v, v, dst_tau[0], dst_tau[1], v, dst_tour, dst_W, dst_col, none)

    assert call(src_col=8) == P.EINVAL          # source columns past its width
    assert call(dst_col=8) == P.EINVAL          # destination columns past its width
    assert call(src_col=-1) == P.EINVAL
    assert call(H=0) == P.EINVAL
    assert call(ncols=-1) == P.EINVAL
    assert call(src_occ=none) == P.EINVAL       # required plane missing
    assert call(src_tau=(v, none)) == P.EINVAL  # pheromone pointers all or none
    assert call(dst_tau=(none, none)) == P.EINVAL
    assert call(dst_tour=none) == P.EINVAL      # tour pointers both or neither
    assert call(ncols=0) == P.OK                # nothing to copy: no launch
