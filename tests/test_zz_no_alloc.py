"""Allocation-free step: sim_step_noalloc, called through the C ABI on device
buffers the caller owns, gives the same results as sim_step.

The entry point exists for callers that cannot let the library allocate
device memory while they run (fixed device-memory budgets, frameworks with
their own caching allocator, work recorded into CUDA graphs): its one piece
of scratch, the proposal plane, lives in a fixed device array of the library.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1412_4933_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_4933_gb300 import pedsim as P  # noqa: E402

CASES = [
    WL.Scenario(176, 80, WL.ACO, 1500, 30, 23, 2, rho=0.1, name="aco_176x80"),
    WL.Scenario(128, 64, WL.LEM, 900, 20, 5, 2, name="lem_128x64"),
    WL.Scenario(96, 48, WL.ACO, 600, 24, 9, 2, rho=0.03, deposit_mode=1, name="aco_inverse_tour"),
    # more cells than one pass of the grid-stride kernels covers (16 CTAs of
    # 256 threads per SM: 622,592 cells on 152 SMs)
    WL.Scenario(1024, 1024, WL.LEM, 60000, 64, 41, 2, name="lem_1024x1024"),
    WL.Scenario(1024, 1024, WL.ACO, 60000, 64, 42, 2, rho=0.05, name="aco_1024x1024"),
]


def _dev(a, dtype=None):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda")


@pytest.mark.parametrize("sc", CASES, ids=lambda s: s.name)
def test_noalloc_matches_sim_step_two_calls_in_a_row(sc):
    prm = P.params_of(sc)
    ref = P.Sim(sc.W, sc.H, prm)
    ref.place(sc.seed)
    g0, a0 = ref.read_grid(), ref.read_agents()
    aco = sc.model == WL.ACO
    occ = [_dev(g0["occ"]), torch.empty_like(_dev(g0["occ"]))]
    ids = _dev(g0["ids"])
    tauA = [_dev(g0["tauA"]), torch.empty_like(_dev(g0["tauA"]))] if aco else [None, None]
    tauB = [_dev(g0["tauB"]), torch.empty_like(_dev(g0["tauB"]))] if aco else [None, None]
    arrival = _dev(a0["arrival"])
    tour = _dev(a0["tour"])
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    for k in range(2):
        rc = P.step_noalloc(sc.W, sc.H, prm, sc.seed, k, occ[k % 2], occ[(k + 1) % 2], ids,
                            tauA[k % 2], tauB[k % 2], tauA[(k + 1) % 2], tauB[(k + 1) % 2],
                            arrival, tour, counters)
        assert rc == P.OK
        ref.step(1)
        torch.cuda.synchronize()
        g, a = ref.read_grid(), ref.read_agents()
        o = occ[(k + 1) % 2].cpu().numpy()
        assert np.array_equal(o, g["occ"]), f"step {k + 1}: occupancy"
        i = ids.cpu().numpy().view(np.uint32)
        assert np.array_equal(np.where(o != 0, i, 0), g["ids"]), f"step {k + 1}: ids"
        if aco:
            for t, name in ((tauA, "tauA"), (tauB, "tauB")):
                got = t[(k + 1) % 2].cpu().numpy().view(np.uint32)
                assert np.array_equal(got, g[name].view(np.uint32)), f"step {k + 1}: {name}"
        assert np.array_equal(arrival.cpu().numpy().view(np.uint32), a["arrival"])
        assert np.array_equal(tour.cpu().numpy().view(np.uint32), a["tour"].view(np.uint32))
        st = ref.stats()
        c = counters.cpu().numpy()
        assert [int(c[0]), int(c[1]), int(c[2]), int(c[3])] == \
            [st["moved"], st["conflicts"], st["crossed"][0], st["crossed"][1]], f"step {k + 1}"
    ref.close()


def test_noalloc_rejects_oversize_grids_and_aliased_buffers():
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    words = torch.zeros(64, dtype=torch.int32, device="cuda")
    # 8192 x 4096 exceeds the 2^24-cell scratch array: rejected before any launch
    big = P.make_params(model=P.LEM, n_per_side=10, band_cols=16)
    assert P.step_noalloc(8192, 4096, big, 1, 0, small, small[1:], words, arrival=words) == P.EINVAL
    assert P.NOALLOC_MAX_CELLS == 1 << 24
    # occupancy in and out must not share a byte: the same buffer, or one
    # starting inside the other, is rejected
    prm = P.make_params(model=P.LEM, n_per_side=10, band_cols=4)
    occ = torch.zeros(512, dtype=torch.uint8, device="cuda")
    assert P.step_noalloc(16, 16, prm, 1, 0, occ, occ, words, arrival=words) == P.EINVAL
    assert P.step_noalloc(16, 16, prm, 1, 0, occ, occ[100:], words, arrival=words) == P.EINVAL
    assert P.step_noalloc(16, 16, prm, 1, 0, occ[100:], occ, words, arrival=words) == P.EINVAL
    # adjacent, disjoint halves of one buffer are accepted (a real step on
    # an empty 16 x 16 grid with buffers of the full sizes)
    ids = torch.zeros(256, dtype=torch.int32, device="cuda")
    arrival = torch.zeros(2 * 10 + 1, dtype=torch.int32, device="cuda")
    assert P.step_noalloc(16, 16, prm, 1, 0, occ[:256], occ[256:], ids, arrival=arrival) == P.OK
    torch.cuda.synchronize()
    assert int(occ[256:].sum()) == 0
