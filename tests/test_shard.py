"""Multi-rank host logic on CPU: two gloo ranks plan the same shards, cover
every image once, slice their containers and reduce the step time (the
decode itself has no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2201_05213_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_plan_covers_every_image_once_and_balances():
    rng = np.random.default_rng(3)
    sizes = [(int(rng.integers(2, 33)) * 16, int(rng.integers(2, 33)) * 16) for _ in range(256)]
    for world in (1, 2, 3, 8):
        plan = shard.plan_shards(sizes, world)
        flat = sorted(i for p in plan for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(shard.image_cost(*sizes[i]) for i in p) for p in plan]
        # LPT: the most loaded rank exceeds the least by at most one image
        assert max(loads) - min(loads) <= max(shard.image_cost(*s) for s in sizes)
    assert shard.plan_shards([], 2) == [[], []]
    big = [(2048, 2048)] + [(1024, 1024)] * 8
    plan = shard.plan_shards(big, 2)
    assert [sum(shard.image_cost(*big[i]) for i in p) for p in plan] == [6 << 20, 6 << 20]


def test_rank_batch_slices_containers():
    lens = [32, 48, 16, 64]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    data = np.arange(offs[-1], dtype=np.int64).astype(np.uint8)
    out, o = shard.rank_batch(data, offs, [3, 1])
    assert list(o) == [0, 64, 112]
    assert np.array_equal(out[:64], data[offs[3]:offs[4]])
    assert np.array_equal(out[64:], data[offs[1]:offs[2]])
    with pytest.raises(ValueError):
        shard.rank_batch(data, np.array([0, 8, 16]), [0])


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = shard.plan_shards(sizes, world)
        plans = [None] * world
        dist.all_gather_object(plans, plan)
        mine = plan[rank]
        t = shard.max_over_ranks(1.5 + rank)
        q.put((rank, plans, mine, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    sizes = [(64, 64)] * 5 + [(128, 96), (32, 512)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, plans, mine, t in res:
        assert plans[0] == plans[1]           # same plan on every rank, nothing exchanged
        assert t == 2.5                       # max over ranks of 1.5 + rank
    assert sorted(res[0][2] + res[1][2]) == list(range(len(sizes)))
