"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to an outside fact: the numpy library's
Philox4x64-10, exact decimal arithmetic, closed forms of the paper's
pheromone equations (Eq. 3-5), exact symmetry of the rules, and brute-force
enumeration of the step's successor distribution (tests/rules_enum.py).
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import oracle as O
from paper_1412_4933_gb300 import workloads as WL
import rules_enum as RE

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# Philox4x64-10 against numpy's library implementation
# --------------------------------------------------------------------------
def _numpy_block(ctr, key):
    """numpy's Philox emits block(counter + 1) first, so start one below."""
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr))
    v = (v - 1) % (1 << 256)
    start = np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    g = np.random.Philox(counter=start, key=np.array(key, dtype=np.uint64))
    return [int(x) for x in g.random_raw(4)]


def test_philox_matches_numpy_library():
    rng = np.random.default_rng(11)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [0, 0]),
             ([2**64 - 1] * 4, [2**64 - 1] * 2), ([12345, 7, 1, 0], [3, 0])]
    for _ in range(300):
        cases.append(([int(x) for x in rng.integers(0, 2**64, size=4, dtype=np.uint64)],
                      [int(x) for x in rng.integers(0, 2**64, size=2, dtype=np.uint64)]))
    for ctr, key in cases:
        assert O.philox4x64_10(ctr, key) == _numpy_block(ctr, key), (ctr, key)


# --------------------------------------------------------------------------
# Heuristic table: eta_i = 1/D_i, D = distance to the point two cells ahead
# --------------------------------------------------------------------------
def _nearest_f32(d: Decimal) -> np.float32:
    f = np.float32(float(d))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    return min(cands, key=lambda c: (abs(Decimal(float(c)) - d), int(c.view(np.uint32)) & 1))


def test_eta_is_correctly_rounded_inverse_distance():
    getcontext().prec = 60
    expected_d2 = {1: 1, 2: 2, 3: 2, 4: 5, 5: 5, 6: 9, 7: 10, 8: 10}
    for i in range(1, 9):
        exact = Decimal(1) / Decimal(expected_d2[i]).sqrt()
        assert np.float32(O.lib().orc_eta(i)) == _nearest_f32(exact), i
    # ranking of Sec. IV.b: #1 nearest, #2=#3 next, #7/#8 farthest
    e = [O.lib().orc_eta(i) for i in range(1, 9)]
    assert e[0] > e[1] == e[2] > e[3] == e[4] > e[5] > e[6] == e[7]


# --------------------------------------------------------------------------
# LEM normal draw: rank distribution from the exact 12-uniform sum
# --------------------------------------------------------------------------
def _rank_table(m, sigma):
    out = np.empty(12 * 65535 + 1, np.int8)
    O.lib().orc_lem_rank_table(m, sigma, out.ctypes.data)
    return out


@pytest.mark.parametrize("sigma_pow2", [0, 1])
def test_lem_rank_thresholds_exhaustive(sigma_pow2):
    s = np.arange(12 * 65535 + 1)
    k_unclamped = np.zeros_like(s)
    for j in range(1, 14):
        k_unclamped += (s >= RE.rank_threshold(j, sigma_pow2)).astype(s.dtype)
    for m in range(1, 9):
        got = _rank_table(m, float(2 ** sigma_pow2)).astype(np.int64)
        assert np.array_equal(got, np.minimum(k_unclamped, m - 1)), m


def test_lem_rank_probabilities_close_to_rounded_normal():
    phi = lambda v: 0.5 * (1 + math.erf(v / math.sqrt(2)))
    for m in (2, 3, 5, 7):
        probs = [float(p) for p in RE.rank_probs(m)]
        assert abs(sum(probs) - 1) < 1e-12
        normal = [phi(0.5)] + [phi(k + 0.5) - phi(k - 0.5) for k in range(1, m - 1)]
        normal.append(1 - phi(m - 1.5))
        for k in range(m):
            # the 12-uniform sum is within 2.1e-3 of the normal CDF at +-0.5
            assert abs(probs[k] - normal[k]) < 2.5e-3, (m, k, probs[k], normal[k])
    p = [float(v) for v in RE.rank_probs(7)]
    assert abs(p[0] - 0.6915) < 2.5e-3 and abs(p[1] - 0.2417) < 2.5e-3


# --------------------------------------------------------------------------
# ACO roulette (Eq. 2): every 24-bit uniform enumerated
# --------------------------------------------------------------------------
def test_aco_roulette_is_proportional_to_weights():
    rng = np.random.default_rng(3)
    for trial in range(4):
        w = np.zeros(9, np.float32)
        avail = rng.uniform(size=7) < 0.7
        avail[trial % 7] = True
        for i in range(2, 9):
            if avail[i - 2]:
                tau = np.float32(rng.uniform(0.0, 5.0))
                w[i] = O.lib().orc_aco_weight(tau, O.lib().orc_eta(i), 1, 1)
        counts = (O.C.c_uint64 * 9)()
        O.lib().orc_aco_histogram(w.ctypes.data_as(O.C.POINTER(O.C.c_float)), counts)
        counts = np.array(counts, dtype=np.float64)
        assert counts[0] == 0 and counts[1] == 0
        S = float(w.astype(np.float64).sum())
        for i in range(2, 9):
            assert abs(counts[i] / 2**24 - float(w[i]) / S) <= 8 * 2**-24, (trial, i)
            if w[i] == 0:
                assert counts[i] == 0


def test_aco_all_zero_weights_defer_to_lem():
    w = np.zeros(9, np.float32)
    for u in (0, 1, 2**23, 2**24 - 1):
        assert O.lib().orc_aco_pick(w.ctypes.data_as(O.C.POINTER(O.C.c_float)), u) == 0


def test_aco_weight_integer_powers():
    L = O.lib()
    for i in range(1, 9):
        e = np.float32(L.orc_eta(i))
        assert L.orc_aco_weight(2.0, e, 3, 1) == np.float32(8.0) * e
        assert L.orc_aco_weight(0.5, e, 1, 2) == np.float32(0.5) * (e * e)
        assert L.orc_aco_weight(7.0, e, 0, 0) == 1.0
        assert L.orc_aco_weight(3.0, e, 1, 0) == 3.0


# --------------------------------------------------------------------------
# Conflict winner: multiply-high splits 2^32 into k near-equal parts
# --------------------------------------------------------------------------
def test_conflict_index_is_fair():
    L = O.lib()
    for k in range(2, 9):
        bounds = [-(-j * 2**32 // k) for j in range(k + 1)]  # ceil(j 2^32 / k)
        for j in range(k):
            assert L.orc_conflict_index(bounds[j], k) == j
            assert L.orc_conflict_index(bounds[j + 1] - 1, k) == j
            assert bounds[j + 1] - bounds[j] in (2**32 // k, -(-2**32 // k))
        assert L.orc_conflict_index(2**32 - 1, k) == k - 1


# --------------------------------------------------------------------------
# Placement: the n band cells with the smallest library-Philox keys
# --------------------------------------------------------------------------
def test_placement_matches_library_philox_selection():
    W, H, band, n, seed = 32, 32, 4, 40, 99
    p = O.make_params(model=0, n_per_side=n, band_cols=band)
    st = O.Oracle(W, H, p, seed).state()
    for g, (x0, x1), first in ((1, (0, band), 1), (2, (W - band, W), n + 1)):
        keys = []
        for y in range(H):
            for x in range(x0, x1):
                c = y * W + x
                keys.append((_numpy_block([c, 0, 3, 0], [seed, 0])[0], c))
        chosen = sorted(c for _, c in sorted(keys)[:n])
        occ = st["occ"].reshape(-1)
        ids = st["ids"].reshape(-1)
        band_cells = [c for _, c in keys]
        assert sorted(c for c in band_cells if occ[c] == g) == chosen
        assert [int(ids[c]) for c in chosen] == list(range(first, first + n))
    assert int((st["occ"] != 0).sum()) == 2 * n


def test_placement_is_uniform_over_band_cells():
    W, H, band, n = 16, 16, 2, 8
    p = O.make_params(model=0, n_per_side=n, band_cols=band)
    freq = np.zeros((H, W))
    seeds = 3000
    for seed in range(seeds):
        freq += O.Oracle(W, H, p, seed).state()["occ"] != 0
    band_freq = np.concatenate([freq[:, :band].ravel(), freq[:, W - band:].ravel()])
    assert freq[:, band:W - band].sum() == 0
    expected = seeds * n / (band * H)
    chi2 = ((band_freq - expected) ** 2 / expected).sum()
    # 64 cells: chi2 with ~62 d.o.f.; 110 is beyond the 0.9999 quantile
    assert chi2 < 110, chi2


# --------------------------------------------------------------------------
# Invariants every step: conservation, exclusivity, ids a permutation
# --------------------------------------------------------------------------
def _check_invariants(st, n_agents, n_side):
    occ, ids = st["occ"], st["ids"]
    assert int((occ == 1).sum()) == n_side and int((occ == 2).sum()) == n_side
    occupied = ids[occ != 0]
    assert sorted(occupied.tolist()) == list(range(1, n_agents + 1))
    assert np.all(ids[occ == 0] == 0)
    assert np.all(occ <= 2)


@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
def test_conservation_exclusivity_every_step(model):
    W, H, n = 64, 48, 500
    p = O.make_params(model=model, n_per_side=n, band_cols=24, rho=0.05)
    o = O.Oracle(W, H, p, 21)
    for t in range(120):
        st = o.state()
        _check_invariants(st, 2 * n, n)
        # ids keep their group
        if t == 0:
            group_of = {int(i): int(g) for i, g in zip(st["ids"][st["occ"] != 0], st["occ"][st["occ"] != 0])}
        else:
            for i, g in zip(st["ids"][st["occ"] != 0], st["occ"][st["occ"] != 0]):
                assert group_of[int(i)] == int(g)
        o.step(1)
    s = o.stats()
    assert s["agents"] == [n, n] and s["step"] == 120
    assert s["moved"] > 0 and s["conflicts"] > 0


# --------------------------------------------------------------------------
# LEM straight line with no opposing agents (Sec. III forward-first)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
def test_straight_line_arrival_times(model):
    W, H, band = 64, 32, 8
    starts = [(1, 0, 2), (1, 3, 6), (1, 7, 10), (2, 63, 14), (2, 58, 18), (2, 40, 22)]
    occ = np.zeros((H, W), np.uint8)
    ids = np.zeros((H, W), np.uint32)
    for a, (g, x, y) in enumerate(starts, 1):
        occ[y, x] = g
        ids[y, x] = a
    p = O.make_params(model=model, n_per_side=3, band_cols=band, rho=0.1)
    o = O.Oracle(W, H, p, 5, state={"occ": occ, "ids": ids})
    for t in range(1, 80):
        o.step(1)
        st = o.state()
        for a, (g, x0, y) in enumerate(starts, 1):
            s = 1 if g == 1 else -1
            dist = (W - 1 - x0) if g == 1 else x0
            x = x0 + s * min(t, dist)
            assert st["ids"][y, x] == a, (t, a)
    arr = o.state()["arrival"]
    for a, (g, x0, y) in enumerate(starts, 1):
        need = max(0, (W - band - x0) if g == 1 else (x0 - band + 1))
        assert arr[a] == need, (a, arr[a], need)
    s = o.stats()
    assert s["parked"] == [3, 3] and s["crossed"] == [3, 3] and s["conflicts"] == 0


# --------------------------------------------------------------------------
# Pheromone: Eq. 3 decay on an empty grid, Eq. 4/5 deposit by one walker
# --------------------------------------------------------------------------
def test_empty_grid_decay_matches_recurrence_and_closed_form():
    W, H, rho, tau0 = 32, 16, 0.1, 1.0
    p = O.make_params(model=1, n_per_side=0, band_cols=4, rho=rho, tau0=tau0)
    o = O.Oracle(W, H, p, 1)
    q = np.float32(1.0) - np.float32(rho)
    tau = np.float32(tau0)
    for t in range(1, 401):
        o.step(1)
        tau = np.float32(tau * q)
        st = o.state()
        assert np.all(st["tauA"].view(np.uint32) == tau.view(np.uint32)), t
        assert np.all(st["tauB"].view(np.uint32) == tau.view(np.uint32)), t
        exact = tau0 * (1.0 - rho) ** t
        assert abs(float(tau) - exact) <= 2 * t * 2**-24 * exact * (1 + 1e-6), t


def test_decay_keeps_subnormals():
    W, H = 16, 16
    p = O.make_params(model=1, n_per_side=0, band_cols=2, rho=0.5, tau0=1.0)
    o = O.Oracle(W, H, p, 1)
    for t in range(1, 152):
        o.step(1)
        v = o.state()["tauA"][3, 5]
        want = 2.0 ** -t if t <= 149 else 0.0
        assert float(v) == want, t


@pytest.mark.parametrize("mode", [0, 1])
def test_single_walker_deposit(mode):
    W, H, rho, dep, tau0 = 48, 16, 0.05, 1.0, 0.5
    x0, y0 = 2, 7
    occ = np.zeros((H, W), np.uint8); ids = np.zeros((H, W), np.uint32)
    occ[y0, x0] = 1; ids[y0, x0] = 1
    p = O.make_params(model=1, n_per_side=1, band_cols=4, rho=rho, tau0=tau0,
                      deposit=dep, deposit_mode=mode)
    o = O.Oracle(W, H, p, 9, state={"occ": occ, "ids": ids})
    q = np.float32(1.0) - np.float32(rho)
    f32 = np.float32
    expect = np.full((H, W), f32(tau0), np.float32)
    steps = W - 1 - x0 + 5
    for s in range(steps):
        o.step(1)
        expect = (expect * q).astype(np.float32)
        if x0 + s + 1 <= W - 1:
            cell = x0 + s + 1
            d = f32(dep) if mode == 0 else f32(1.0) / f32(s + 1)
            expect[y0, cell] = f32(expect[y0, cell] + d)
        st = o.state()
        assert np.array_equal(st["tauA"].view(np.uint32), expect.view(np.uint32)), s
        decay_only = f32(tau0)
        for _ in range(s + 1):
            decay_only = f32(decay_only * q)
        assert np.all(st["tauB"] == decay_only)
    if mode == 1:
        assert o.state()["tour"][1] == np.float32(W - 1 - x0)


# --------------------------------------------------------------------------
# Exact mirror symmetry: point reflection through the grid centre swaps the
# groups and keeps every rule (test-only mirror mode remaps the RNG cell word
# and reverses the fixed claimant order).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
def test_point_mirror_symmetry_exact(model):
    W, H, n, seed = 64, 48, 400, 77
    p = O.make_params(model=model, n_per_side=n, band_cols=20, rho=0.03)
    a = O.Oracle(W, H, p, seed)
    b = O.Oracle(W, H, p, seed, mirror=True)
    N = 2 * n

    def mirrored(st):
        occ = st["occ"][::-1, ::-1].copy()
        occ = np.where(occ == 1, 2, np.where(occ == 2, 1, 0)).astype(np.uint8)
        ids = st["ids"][::-1, ::-1].copy()
        ids = np.where(ids != 0, N + 1 - ids, 0).astype(np.uint32)
        arr = st["arrival"].copy()
        arr[1:] = st["arrival"][1:][::-1]
        return occ, ids, st["tauB"][::-1, ::-1], st["tauA"][::-1, ::-1], arr

    for t in range(150):
        sa, sb = a.state(), b.state()
        occ, ids, tA, tB, arr = mirrored(sa)
        assert np.array_equal(sb["occ"], occ), t
        assert np.array_equal(sb["ids"], ids), t
        assert np.array_equal(sb["tauA"].view(np.uint32), tA.view(np.uint32)), t
        assert np.array_equal(sb["tauB"].view(np.uint32), tB.view(np.uint32)), t
        assert np.array_equal(sb["arrival"], arr), t
        a.step(1); b.step(1)
    sa, sb = a.stats(), b.stats()
    assert sa["crossed"] == sb["crossed"][::-1] and sa["moved"] == sb["moved"]
    assert sa["conflicts"] == sb["conflicts"] and sa["moved"] > 1000


# --------------------------------------------------------------------------
# 8x8 brute force: successors are legal; for few agents their frequencies
# match the exactly enumerated distribution.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
def test_dense_8x8_successors_are_legal(model):
    W = H = 16  # the smallest legal grid; agents confined to an 8x8 window
    rng = np.random.default_rng(4)
    p = O.make_params(model=model, n_per_side=1, band_cols=2, rho=0.05)
    for trial in range(60):
        win_occ, _ = WL.random_occupancy(8, 8, rng.uniform(0.2, 0.7), 1000 + trial)
        occ = np.zeros((H, W), np.uint8)
        ox, oy = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        if trial % 3 == 0:
            ox, oy = (0 if trial % 2 else 8), (0 if trial % 4 else 8)  # touch the walls
        occ[oy:oy + 8, ox:ox + 8] = win_occ
        ids = np.zeros((H, W), np.uint32)
        nz = np.flatnonzero(occ)
        ids.reshape(-1)[nz] = rng.permutation(len(nz)).astype(np.uint32) + 1
        tau = [rng.uniform(0, 2, size=(H, W)).astype(np.float32) for _ in range(2)]
        o = O.Oracle(W, H, p, 500 + trial, state={"occ": occ, "ids": ids,
                                                  "tauA": tau[0], "tauB": tau[1]}, step=trial)
        o.step(1)
        st = o.state()
        problems = RE.check_successor(occ, ids, st["occ"], st["ids"], model, tau)
        assert not problems, (trial, problems)


def _few_agent_cases():
    cases = []
    # A blocked head-on by B: both must sidestep; a third agent competes.
    occ = np.zeros((16, 16), np.uint8)
    occ[5, 6] = 1; occ[5, 7] = 2; occ[4, 8] = 2
    cases.append(occ)
    # against the top wall, two A agents in a column blocked by a B wall-hugger
    occ = np.zeros((16, 16), np.uint8)
    occ[0, 3] = 1; occ[0, 4] = 2; occ[1, 4] = 2
    cases.append(occ)
    # three A agents in a row: the rear two are blocked
    occ = np.zeros((16, 16), np.uint8)
    occ[8, 2] = 1; occ[8, 3] = 1; occ[8, 4] = 1
    cases.append(occ)
    return cases


@pytest.mark.parametrize("model", [WL.LEM, WL.ACO])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_few_agent_successor_frequencies(model, case):
    scipy_stats = pytest.importorskip("scipy.stats")
    occ = _few_agent_cases()[case]
    H, W = occ.shape
    ids = np.zeros((H, W), np.uint32)
    nz = np.flatnonzero(occ)
    ids.reshape(-1)[nz] = np.arange(1, len(nz) + 1, dtype=np.uint32)
    rng = np.random.default_rng(case)
    tau = [rng.uniform(0.1, 3, size=(H, W)).astype(np.float32) for _ in range(2)]
    exact = RE.successor_distribution(occ, ids, model, tau)
    assert abs(sum(exact.values()) - 1) < 1e-9
    p = O.make_params(model=model, n_per_side=2, band_cols=2, rho=0.05)
    counts = {}
    n_seeds = 20000
    for seed in range(n_seeds):
        o = O.Oracle(W, H, p, seed * 7919 + case,
                     state={"occ": occ, "ids": ids, "tauA": tau[0], "tauB": tau[1]})
        o.step(1)
        st = o.state()
        key = st["occ"].tobytes() + st["ids"].tobytes()
        assert key in exact, "successor outside the enumerated support"
        counts[key] = counts.get(key, 0) + 1
    keys = sorted(exact, key=lambda k: -exact[k])
    obs, exp, rest_o, rest_e = [], [], 0, 0.0
    for k in keys:
        e = exact[k] * n_seeds
        if e >= 5:
            obs.append(counts.get(k, 0)); exp.append(e)
        else:
            rest_o += counts.get(k, 0); rest_e += e
    if rest_e > 0:
        obs.append(rest_o); exp.append(rest_e)
    exp = np.array(exp) * (sum(obs) / sum(exp))
    if len(obs) > 1:
        assert scipy_stats.chisquare(obs, exp).pvalue > 1e-4


# --------------------------------------------------------------------------
# Parameter validation
# --------------------------------------------------------------------------
def test_parameter_validation():
    L = O.lib()
    ok = O.make_params(model=1, n_per_side=10, band_cols=4)
    assert L.orc_check_params(64, 64, O.C.byref(ok)) == 0
    bad = [(60, 64, ok), (64, 8, ok),
           (64, 64, O.make_params(model=1, n_per_side=10, band_cols=33)),
           (64, 64, O.make_params(model=1, n_per_side=257, band_cols=4)),
           (64, 64, O.make_params(model=1, n_per_side=10, band_cols=4, rho=0.0)),
           (64, 64, O.make_params(model=1, n_per_side=10, band_cols=4, rho=1.5)),
           (64, 64, O.make_params(model=1, n_per_side=10, band_cols=4, alpha=5)),
           (64, 64, O.make_params(model=2, n_per_side=10, band_cols=4)),
           (64, 64, O.make_params(model=0, n_per_side=10, band_cols=0))]
    for W, H, prm in bad:
        assert L.orc_check_params(W, H, O.C.byref(prm)) != 0, (W, H)


# --------------------------------------------------------------------------
# Eq. 5 tour length with diagonal moves: L_k grows by 1 per orthogonal move
# and by fl(sqrt 2) per diagonal one, before the deposit 1/L_k (Sec. IV.d)
# --------------------------------------------------------------------------
def _f32_sqrt2_from_decimal():
    getcontext().prec = 60
    return _nearest_f32(Decimal(2).sqrt())


def test_diagonal_step_tour_is_rounded_sqrt2():
    # An A agent one column before its goal edge, its forward cell held by a
    # parked A agent: forward is blocked for good, so it moves sideways or
    # diagonally (a forward diagonal parks it).  Over seeds where that first
    # move is diagonal, the tour must be fl(sqrt 2) and the deposit fl(1/L)
    # on top of the evaporated value.
    W, H, y = 32, 16, 8
    rho, tau0 = 0.05, 0.75
    sqrt2 = _f32_sqrt2_from_decimal()
    f32 = np.float32
    q = f32(1.0) - f32(rho)
    diag_seen = orth_seen = 0
    for seed in range(60):
        occ = np.zeros((H, W), np.uint8); ids = np.zeros((H, W), np.uint32)
        occ[y, W - 2] = 1; ids[y, W - 2] = 1    # the walker
        occ[y, W - 1] = 1; ids[y, W - 1] = 2    # parked on the goal column
        p = O.make_params(model=1, n_per_side=1, band_cols=4, rho=rho, tau0=tau0,
                          deposit_mode=1)
        o = O.Oracle(W, H, p, seed, state={"occ": occ, "ids": ids})
        o.step(1)
        st = o.state()
        (ny,), (nx,) = np.nonzero(st["ids"] == 1)
        dx, dy = nx - (W - 2), ny - y
        if dx == 0 and dy == 0:
            continue
        if dx != 0 and dy != 0:
            diag_seen += 1
            assert st["tour"][1] == sqrt2, seed
            want = f32(f32(f32(tau0) * q) + f32(f32(1.0) / sqrt2))
        else:
            orth_seen += 1
            assert st["tour"][1] == f32(1.0), seed
            want = f32(f32(f32(tau0) * q) + f32(1.0))
        assert st["tauA"][ny, nx].view(np.uint32) == want.view(np.uint32), seed
    # the forward diagonals are the most likely ranks of Eq. 2
    assert diag_seen >= 20 and orth_seen >= 1, (diag_seen, orth_seen)


def test_tour_and_deposit_follow_the_moves_of_a_dense_run():
    # Dense ACO run with Eq. 5 deposits: from the ids plane of consecutive
    # states, recompute every agent's tour (1 per orthogonal and fl(sqrt 2)
    # per diagonal move, summed in move order) and both pheromone planes
    # (evaporate every cell, then add fl(1/L) of each mover at its new cell).
    W, H, n, rho = 48, 32, 300, 0.07
    sqrt2 = _f32_sqrt2_from_decimal()
    f32 = np.float32
    q = f32(1.0) - f32(rho)
    p = O.make_params(model=1, n_per_side=n, band_cols=16, rho=rho, tau0=1.0,
                      deposit_mode=1)
    o = O.Oracle(W, H, p, 31)
    st = o.state()
    N = 2 * n
    pos = np.zeros((N + 1, 2), np.int64)
    for yy, xx in zip(*np.nonzero(st["ids"])):
        pos[st["ids"][yy, xx]] = (xx, yy)
    tour = np.zeros(N + 1, np.float32)
    tau = [st["tauA"].copy(), st["tauB"].copy()]
    group = np.zeros(N + 1, np.int64)
    group[st["ids"][st["occ"] != 0]] = st["occ"][st["occ"] != 0]
    diag_moves = 0
    for t in range(80):
        o.step(1)
        nxt = o.state()
        tau = [(tp * q).astype(np.float32) for tp in tau]
        for yy, xx in zip(*np.nonzero(nxt["ids"])):
            a = nxt["ids"][yy, xx]
            dx, dy = xx - pos[a][0], yy - pos[a][1]
            if dx == 0 and dy == 0:
                continue
            assert max(abs(dx), abs(dy)) == 1, (t, a)
            diag = dx != 0 and dy != 0
            diag_moves += diag
            tour[a] = f32(tour[a] + (sqrt2 if diag else f32(1.0)))
            g = group[a] - 1
            tau[g][yy, xx] = f32(tau[g][yy, xx] + f32(f32(1.0) / tour[a]))
            pos[a] = (xx, yy)
        assert np.array_equal(nxt["tour"].view(np.uint32), tour.view(np.uint32)), t
        assert np.array_equal(nxt["tauA"].view(np.uint32), tau[0].view(np.uint32)), t
        assert np.array_equal(nxt["tauB"].view(np.uint32), tau[1].view(np.uint32)), t
    assert diag_moves > 200, diag_moves


# --------------------------------------------------------------------------
# Conflict counter (Sec. IV.d): the number of (cell, step) pairs with two or
# more claimants -- cells, not losing agents
# --------------------------------------------------------------------------
def test_head_on_conflict_one_winner_each_side_half_the_time():
    W, H, x, y = 32, 16, 10, 6
    wins = 0
    seeds = 400
    for seed in range(seeds):
        occ = np.zeros((H, W), np.uint8); ids = np.zeros((H, W), np.uint32)
        occ[y, x] = 1; ids[y, x] = 1          # A heading +x
        occ[y, x + 2] = 2; ids[y, x + 2] = 2  # B heading -x: both forward into x+1
        p = O.make_params(model=0, n_per_side=1, band_cols=4)
        o = O.Oracle(W, H, p, seed, state={"occ": occ, "ids": ids})
        o.step(1)
        s, st = o.stats(), o.state()
        assert s["moved"] == 1 and s["conflicts"] == 1, (seed, s)
        winner = int(st["ids"][y, x + 1])
        assert winner in (1, 2)
        loser_cell = (y, x + 2) if winner == 1 else (y, x)
        assert st["ids"][loser_cell] == 3 - winner  # the loser stays
        wins += winner == 1
    # binomial(400, 1/2): 4.5 standard deviations either side
    assert abs(wins - seeds / 2) < 4.5 * math.sqrt(seeds / 4), wins


def test_conflict_counter_counts_cells_not_losers():
    # Dense random states: every agent's decision at the step is taken from
    # the oracle's own decision hook, then the claimants of every empty cell
    # are counted here.  moved must be the number of claimed cells and
    # conflicts the number of cells with >= 2 claimants; states with three
    # or more claimants on one cell make the two readings differ.
    W, H = 32, 32
    rng = np.random.default_rng(8)
    k3_cells = 0
    for trial in range(40):
        model = trial % 2
        occ, _ = WL.random_occupancy(H, W, rng.uniform(0.3, 0.6), 300 + trial)
        ids = np.zeros((H, W), np.uint32)
        nz = np.flatnonzero(occ)
        ids.reshape(-1)[nz] = rng.permutation(len(nz)).astype(np.uint32) + 1
        tau = [rng.uniform(0.1, 2, size=(H, W)).astype(np.float32) for _ in range(2)]
        p = O.make_params(model=model, n_per_side=1, band_cols=2, rho=0.05)
        o = O.Oracle(W, H, p, 900 + trial, state={"occ": occ, "ids": ids, "tauA": tau[0],
                                                  "tauB": tau[1]}, step=trial)
        claims = {}
        for yy, xx in zip(*np.nonzero(occ)):
            i = o.decide_at(int(xx), int(yy))
            if i == 0:
                continue
            s = 1 if occ[yy, xx] == 1 else -1
            fx, fy = RE.FRAME[i]
            tgt = (int(yy) + s * fy, int(xx) + s * fx)
            claims[tgt] = claims.get(tgt, 0) + 1
        o.step(1)
        st = o.stats()
        assert st["moved"] == len(claims), trial
        assert st["conflicts"] == sum(1 for k in claims.values() if k >= 2), trial
        k3_cells += sum(1 for k in claims.values() if k >= 3)
    assert k3_cells >= 10, k3_cells
