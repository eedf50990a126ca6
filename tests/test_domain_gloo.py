"""Domain decomposition, host side, on CPU: the column partition and the
halo exchange between ranks (gloo, world sizes 2 and 3).

Every rank holds one strip of a synthetic whole-grid state: its interior
columns correct, its halo columns and the per-agent entries of every agent
outside its interior wrong.  After one exchange each rank's halo columns
(occupancy, ids, both pheromone planes) and the arrival step and tour length
of every agent standing in them must equal the whole grid's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1412_4933_gb300 import domain as D


def test_partition_and_layout():
    assert D.partition(48, 3) == [(0, 16), (16, 32), (32, 48)]
    assert D.partition(50, 3) == [(0, 17), (17, 34), (34, 50)]
    with pytest.raises(ValueError):
        D.partition(8, 3)  # strips narrower than the halo
    lay = D.StripLayout(48, 16, 32)
    assert (lay.ea, lay.eb, lay.width, lay.lo, lay.hi) == (13, 35, 22, 3, 19)
    assert lay.left_halo() == (13, 16) and lay.right_halo() == (32, 35)
    first, last = D.StripLayout(48, 0, 16), D.StripLayout(48, 32, 48)
    assert (first.ea, first.eb, first.lo) == (0, 19, 0)
    assert (last.ea, last.eb, last.hi) == (29, 48, 19)


def global_state(W, H, n, seed):
    rng = np.random.default_rng(seed)
    occ = np.zeros((H, W), np.uint8)
    cells = rng.choice(W * H, size=2 * n, replace=False)
    occ.reshape(-1)[cells] = rng.integers(1, 3, size=2 * n)
    ids = np.zeros((H, W), np.int32)
    ids.reshape(-1)[cells] = rng.permutation(2 * n) + 1
    # stale ids at some empty cells (the kernels leave them behind)
    empty = np.flatnonzero(occ.reshape(-1) == 0)[:10]
    ids.reshape(-1)[empty] = rng.integers(1, 2 * n + 1, size=len(empty))
    tau = [rng.uniform(0, 2, size=(H, W)).astype(np.float32) for _ in range(2)]
    arrival = rng.integers(0, 500, size=2 * n + 1).astype(np.int32)
    tour = rng.uniform(0, 90, size=2 * n + 1).astype(np.float32)
    return occ, ids, tau, arrival, tour


def _worker(rank, world, port, W, H, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        occ, ids, tau, arrival, tour = global_state(W, H, n, 5)
        layouts = [D.StripLayout(W, a, b) for a, b in D.partition(W, world)]
        lay = layouts[rank]
        st = D.StripState(torch, lay, H, 2 * n, True, "cpu")
        # interior correct; halo and foreign agents wrong
        cols = slice(lay.ea, lay.eb)
        st.occ[0].copy_(torch.from_numpy(np.where(True, 0, occ[:, cols]).astype(np.uint8)))
        st.ids.fill_(0)
        for t in (st.tau[0][0], st.tau[1][0]):
            t.fill_(-1.0)
        inner = slice(lay.lo, lay.hi)
        st.occ[0][:, inner] = torch.from_numpy(occ[:, lay.a:lay.b].copy())
        st.ids[:, inner] = torch.from_numpy(ids[:, lay.a:lay.b].copy())
        st.tau[0][0][:, inner] = torch.from_numpy(tau[0][:, lay.a:lay.b].copy())
        st.tau[1][0][:, inner] = torch.from_numpy(tau[1][:, lay.a:lay.b].copy())
        mine = ids[:, lay.a:lay.b][occ[:, lay.a:lay.b] != 0]
        st.arrival.fill_(-7)
        st.tour.fill_(-7.0)
        st.arrival[torch.from_numpy(mine.astype(np.int64))] = torch.from_numpy(arrival[mine])
        st.tour[torch.from_numpy(mine.astype(np.int64))] = torch.from_numpy(tour[mine])
        D.DistExchange(dist, st, rank, world, layouts).exchange(0)
        # every local column now equals the whole grid's
        ok_planes = (np.array_equal(st.occ[0].numpy(), occ[:, cols])
                     and np.array_equal(np.where(occ[:, cols] != 0, st.ids.numpy(), 0),
                                        np.where(occ[:, cols] != 0, ids[:, cols], 0))
                     and np.array_equal(st.tau[0][0].numpy(), tau[0][:, cols])
                     and np.array_equal(st.tau[1][0].numpy(), tau[1][:, cols]))
        local_agents = ids[:, cols][occ[:, cols] != 0]
        ok_agents = (np.array_equal(st.arrival.numpy()[local_agents], arrival[local_agents])
                     and np.array_equal(st.tour.numpy()[local_agents], tour[local_agents]))
        halo_agents = len(local_agents) - len(mine)
        q.put((rank, ok_planes, ok_agents, halo_agents))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_with_gloo(world):
    W, H, n = 48, 32, 300
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    procs = [ctx.Process(target=_worker, args=(r, world, port, W, H, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_planes, ok_agents, halo_agents in out:
        assert ok_planes, f"rank {rank}: halo planes differ from the whole grid"
        assert ok_agents, f"rank {rank}: per-agent entries of halo agents differ"
        assert halo_agents > 0, rank


@pytest.mark.parametrize("n_strips", [2, 3])
def test_local_exchange_on_cpu(n_strips):
    """LocalExchange between strips held by one process (CPU tensors: the
    packed-slab path, used between devices): after one exchange every
    strip's local columns and the entries of every agent on them equal the
    whole grid's; agents elsewhere keep their (stale) entries."""
    W, H, n = 48, 20, 150
    occ, ids, tau, arrival, tour = global_state(W, H, n, 9)
    layouts = [D.StripLayout(W, a, b) for a, b in D.partition(W, n_strips)]
    strips = []
    for lay in layouts:
        st = D.StripState(torch, lay, H, 2 * n, True, "cpu")
        st.occ[0].fill_(0)
        st.ids.fill_(0)
        for t in (st.tau[0][0], st.tau[1][0]):
            t.fill_(-1.0)
        inner = slice(lay.lo, lay.hi)
        st.occ[0][:, inner] = torch.from_numpy(occ[:, lay.a:lay.b].copy())
        st.ids[:, inner] = torch.from_numpy(ids[:, lay.a:lay.b].copy())
        st.tau[0][0][:, inner] = torch.from_numpy(tau[0][:, lay.a:lay.b].copy())
        st.tau[1][0][:, inner] = torch.from_numpy(tau[1][:, lay.a:lay.b].copy())
        mine = ids[:, lay.a:lay.b][occ[:, lay.a:lay.b] != 0].astype(np.int64)
        st.arrival.fill_(-7)
        st.tour.fill_(-7.0)
        st.arrival[torch.from_numpy(mine)] = torch.from_numpy(arrival[mine])
        st.tour[torch.from_numpy(mine)] = torch.from_numpy(tour[mine])
        strips.append(st)
    D.LocalExchange(strips).exchange(0)
    halo_agents = 0
    for lay, st in zip(layouts, strips):
        cols = slice(lay.ea, lay.eb)
        assert np.array_equal(st.occ[0].numpy(), occ[:, cols])
        on = occ[:, cols] != 0
        assert np.array_equal(st.ids.numpy()[on], ids[:, cols][on])
        assert np.array_equal(st.tau[0][0].numpy(), tau[0][:, cols])
        assert np.array_equal(st.tau[1][0].numpy(), tau[1][:, cols])
        local = ids[:, cols][on]
        assert np.array_equal(st.arrival.numpy()[local], arrival[local])
        assert np.array_equal(st.tour.numpy()[local], tour[local])
        others = np.setdiff1d(np.arange(1, 2 * n + 1), local)
        assert (st.arrival.numpy()[others] == -7).all()
        halo_agents += len(local) - int((occ[:, lay.a:lay.b] != 0).sum())
    assert halo_agents > 0  # some agents stood in the halos
