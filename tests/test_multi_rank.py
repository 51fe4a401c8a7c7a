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


def _split_worker(rank, world, port, q):
    """One rank of a simulation split over two ranks, on CPU: the layout this rank's context
    would own (host-only), and the all-reduce of field parts."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        from paper_2311_05170_gb300 import native
        from paper_2311_05170_gb300.shard import reduce_fields
        w = W.config_graded(nsteps=1)
        s = native.Solver(w, host_only=True, rank=rank, nranks=world)
        mine = []
        j = 0
        while True:
            try:
                info = s.debug_system(j)
            except native.TpnsError:
                break
            mine.append((int(info["node"].min()), len(info["node"]), int(info["comp"].max())))
            j += 1
        s.close()
        sig = gather_lists(mine, True)
        parts = {"a": np.arange(5, dtype=np.float64) * (rank + 1), "b": np.full(3, float(rank))}
        tot = reduce_fields(parts, True)
        q.put((rank, mine, sig, {k: v.tolist() for k, v in tot.items()}))
    finally:
        dist.destroy_process_group()


def test_one_simulation_split_over_two_gloo_ranks():
    """The two ranks' subdomain sets are disjoint and together are the whole partition (as the
    library builds it on each rank without communicating), the Oseen / Darcy split is even, and
    the field parts sum to the whole field on every rank."""
    from paper_2311_05170_gb300 import native, build
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = native.Solver(W.config_graded(nsteps=1), host_only=True)
    full = []
    j = 0
    while True:
        try:
            info = s.debug_system(j)
        except native.TpnsError:
            break
        full.append((int(info["node"].min()), len(info["node"]), int(info["comp"].max())))
        j += 1
    s.close()
    a, b = res[0][1], res[1][1]
    assert sorted(a + b) == sorted(full) and not set(a) & set(b)
    for r in res:
        assert sorted(r[2]) == sorted(full)        # the all-gathered view is the same on both ranks
        assert r[3]["a"] == [0.0, 3.0, 6.0, 9.0, 12.0] and r[3]["b"] == [1.0, 1.0, 1.0]
    # 16 Oseen systems (comp max 2) and 16 porous problems, split 8 / 8 each
    for part in (a, b):
        assert sum(1 for x in part if x[2] == 2) == 8 and sum(1 for x in part if x[2] == 0) == 8


def test_split_refuses_more_ranks_than_subdomains():
    from paper_2311_05170_gb300 import native, build
    build.build()
    with pytest.raises(native.TpnsError):
        native.Solver(W.config_small(nsteps=1), host_only=True, rank=0, nranks=5)
