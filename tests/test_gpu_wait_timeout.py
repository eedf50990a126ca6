"""Failure detection on the GPU without a fault: a bounded device wait is
made to run out on purpose and reported as PEDSIM_ETIMEDOUT.

The tiled resolution kernel waits (bounded) for its TMA copies.  The test
hook sim_set_wait_test shortens that bound and makes the kernel issue no
copy at all, so nothing ever completes the wait: each CTA gives up after the
bound, returns without writing state and with nothing in flight, and the
handle's error word is set.  No trap, fault or unbounded wait is involved;
afterwards the CUDA context must still run a scenario bit-exactly."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1412_4933_gb300 import pedsim
    return pedsim


def _params(P):
    return P.make_params(model=P.ACO, n_per_side=120, band_cols=8, rho=0.05)


def test_wait_runs_out_and_reports_timeout(P):
    import torch
    sim = P.Sim(64, 32, _params(P))
    sim.set_variant(P.VARIANT_TILED)
    sim.place(5)
    sim.step(3)
    assert sim.device_status() == 0
    # about 0.5 ms of SM clock instead of the default ~2 s
    sim.set_wait_test(wait_cycles=1 << 20, flags=P.TEST_SKIP_RESOLVE_LOADS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(1)
    status = sim.device_status()
    dt = time.perf_counter() - t0
    assert status == P.ETIMEDOUT
    assert dt < 1.0, f"the short wait limit was not used ({dt:.3f} s)"
    assert sim.device_status() == 0  # reading the status cleared it
    sim.close()
    torch.cuda.synchronize()


def test_unknown_test_flag_is_rejected(P):
    sim = P.Sim(64, 32, _params(P))
    with pytest.raises(P.PedsimError) as e:
        sim.set_wait_test(0, 2)
    assert e.value.code == P.EINVAL
    sim.close()


def test_context_usable_after_timeout_and_limit_honoured_when_met(P):
    from oracle import oracle as O
    import torch
    # a timed-out step first ...
    bad = P.Sim(64, 32, _params(P))
    bad.set_variant(P.VARIANT_TILED)
    bad.place(6)
    bad.set_wait_test(wait_cycles=1 << 20, flags=P.TEST_SKIP_RESOLVE_LOADS)
    bad.step(2)
    assert bad.device_status() == P.ETIMEDOUT
    bad.close()
    # ... then a fresh scenario with a short limit that its copies meet runs
    # bit-exactly against the oracle
    kw = dict(model=P.ACO, n_per_side=120, band_cols=8, rho=0.05)
    sim = P.Sim(64, 32, P.make_params(**kw))
    sim.set_variant(P.VARIANT_TILED)
    sim.set_wait_test(wait_cycles=1 << 24, flags=0)
    sim.place(6)
    orc = O.Oracle(64, 32, O.make_params(**kw), 6)
    for t in range(12):
        sim.step(1)
        orc.step(1)
        g, o = sim.read_grid(), orc.state()
        assert np.array_equal(g["occ"], o["occ"]), t
        assert np.array_equal(g["ids"], o["ids"]), t
        assert np.array_equal(g["tauA"].view(np.uint32), o["tauA"].view(np.uint32)), t
    assert sim.device_status() == 0
    sim.close()
    torch.cuda.synchronize()
