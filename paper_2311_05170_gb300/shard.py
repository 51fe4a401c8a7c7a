"""Multi-GPU layouts.

Within one time step the local problems of the two-grid method (Algorithm 3) are coupled
only through the coarse solve that precedes them and the glue that follows.  Two layouts:

* independent simulations per rank (replicas of one workload, or the requests of a serving
  workload), with no data-path collective; the collectives run after a timed region, to
  reduce timings and statistics (max of the per-rank times, sums of the units processed, the
  pooled list of per-step latencies);
* one simulation split over ranks (tpns_options.rank / nranks): every rank repeats the
  coarse solve, solves its own subdomains (assigned by estimated work inside the library, the
  same on every rank) and returns its part of the glued field; the glued field of Step 4 is
  the sum of the parts, so the only exchange is one sum (all-reduce) of the fields, and only
  when a global field is wanted.

Every function takes the process group explicitly (None = a single process), so the same
code runs on NCCL with CUDA tensors and on gloo with CPU tensors.
"""
import heapq


def request_work(w, nsteps):
    """Work estimate of one simulation: fine cells of both regions times time steps."""
    cols = w.nx_coarse * w.fine_per_coarse_x
    rows = sum(w.fine_rows_from_gamma[: w.ny_coarse])
    return 2 * cols * rows * nsteps


def shard_requests(requests, rank, world):
    """This rank's share of `requests` (list of (arrival, Workload, nsteps)).

    Longest-processing-time-first assignment by request_work, ties broken by index, so every
    rank computes the same partition without communicating; the shares are disjoint, cover
    all requests and keep their arrival order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    order = sorted(range(len(requests)), key=lambda i: (-request_work(requests[i][1], requests[i][2]), i))
    heap = [(0, r) for r in range(world)]
    owner = {}
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + request_work(requests[i][1], requests[i][2]), r))
    return [requests[i] for i in range(len(requests)) if owner[i] == rank]


def _reduce(value, group, op, device):
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op, group=group)
    return float(t.item())


def max_over_ranks(value, dist_on, device="cpu", group=None):
    """Largest value over the ranks (the whole job's time is its slowest rank's)."""
    if not dist_on:
        return float(value)
    import torch.distributed as dist
    return _reduce(value, group, dist.ReduceOp.MAX, device)


def sum_over_ranks(value, dist_on, device="cpu", group=None):
    """Sum over the ranks (units processed by the whole job)."""
    if not dist_on:
        return float(value)
    import torch.distributed as dist
    return _reduce(value, group, dist.ReduceOp.SUM, device)


def gather_lists(values, dist_on, group=None):
    """Concatenation of every rank's list, in rank order (per-step latencies for p50/p99)."""
    if not dist_on:
        return list(values)
    import torch.distributed as dist
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, list(values), group=group)
    return [x for part in out for x in part]


def reduce_fields(parts, dist_on, device="cpu", group=None):
    """Glued fields of a simulation split over ranks: the sum over ranks of each rank's part
    (dict field -> 1D float64 array); every rank gets the whole field."""
    if not dist_on:
        return {k: v.copy() for k, v in parts.items()}
    import numpy as np
    import torch
    import torch.distributed as dist
    out = {}
    for k in sorted(parts):
        t = torch.from_numpy(np.ascontiguousarray(parts[k])).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out[k] = t.cpu().numpy()
    return out
