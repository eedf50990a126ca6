"""Multi-process host logic on CPU (gloo, world size 2): the benchmark's
max-over-ranks timing and the sharding of independent scenarios across ranks.
Every run here has one GPU, so the N-GPU path is replicas/shards with no
collective on the data path; these tests cover the host side of it."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1412_4933_gb300 import workloads as WL
        t = bench.max_over_ranks(1.5 + rank, dist)
        scs = WL.batched_scenarios(count=37, steps=10)
        mine = WL.shard(scs, rank, world)
        names = [None] * world
        dist.all_gather_object(names, [s.name for s in mine])
        q.put((rank, t, names))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_sharding_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, names in out:
        assert t == 2.5  # max of 1.5 and 2.5 on every rank
        flat = [n for part in names for n in part]
        assert sorted(flat) == sorted(f"batch{i}" for i in range(37))
        assert len(set(flat)) == 37


def test_shard_rejects_bad_ranks():
    from paper_1412_4933_gb300 import workloads as WL
    with pytest.raises(ValueError):
        WL.shard([1, 2], 2, 2)
    assert WL.shard(range(5), 1, 2) == [1, 3]
