"""Multi-GPU host logic on CPU: two gloo ranks shard serving requests without talking to each
other, then reduce timings and pool latencies the way the bench does on NCCL."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2311_05170_gb300.shard import (gather_lists, max_over_ranks, request_work, shard_requests,
                                          sum_over_ranks)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs = [(a, w, 100) for a, w in W.serving_requests(n=64)]
        mine = shard_requests(reqs, rank, world)
        names = gather_lists([w.name for _, w, _ in mine], True)
        work = sum(request_work(w, n) for _, w, n in mine)
        loads = gather_lists([work], True)
        t = max_over_ranks(1.5 + rank, True)
        units = sum_over_ranks(10 * (rank + 1), True)
        lat = gather_lists([rank * 100.0 + i for i in range(3)], True)
        q.put((rank, names, loads, t, units, lat, [w.name for _, w, _ in mine]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    all_names = [w.name for _, w in W.serving_requests(n=64)]
    for rank, names, loads, t, units, lat, mine in res:
        # every rank saw the same pooled view
        assert sorted(names) == sorted(all_names) and len(names) == len(set(names))
        assert t == 2.5 and units == 30.0
        assert lat == [0.0, 1.0, 2.0, 100.0, 101.0, 102.0]
        # balanced: the heavier rank carries at most one largest request more
        biggest = max(request_work(w, 100) for _, w in W.serving_requests(n=64))
        assert abs(loads[0] - loads[1]) <= biggest
    # the shares are disjoint and in arrival order
    a, b = res[0][6], res[1][6]
    assert not set(a) & set(b)
    order = {n: i for i, n in enumerate(all_names)}
    assert a == sorted(a, key=order.get) and b == sorted(b, key=order.get)


def test_single_process_helpers_need_no_group():
    reqs = W.serving_requests_small(n=5)
    assert shard_requests(reqs, 0, 1) == reqs
    assert max_over_ranks(3.0, False) == 3.0 and sum_over_ranks(4.0, False) == 4.0
    assert gather_lists([1, 2], False) == [1, 2]
    with pytest.raises(ValueError):
        shard_requests(reqs, 2, 2)
