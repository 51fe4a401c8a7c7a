"""Serving loop for many simulations of the two-grid method on one GPU (continuous batching).

Requests arrive over time (Poisson arrivals); each is a simulation with its own mesh sizes and
physical parameters.  A request is admitted when the device memory it needs fits in the HBM
budget left by the simulations on the device (the library refuses a context whose footprint
exceeds the budget it is given: TPNS_EBUDGET); its coarse and fine state and its Darcy factors
then stay resident until it has run its steps.  Every scheduler tick advances all admitted
simulations by one time step with one tpns_batch_step call: their steps are enqueued side by
side on their own streams, so their work overlaps on the device.  Finished simulations are
released at once, which frees memory for waiting ones.

The per-step latency of a simulation is the device time of its step within the tick, from the
step's start on the simulation's stream to its end, with the other simulations running beside
it (tpns_stats.last_step_ms); the tick itself ends when the slowest step ends (tick_ms).
"""
import time

import numpy as np

from .native import TPNS_EBUDGET, Solver, TpnsError, batch_step


class Request:
    def __init__(self, rid, arrival, workload, nsteps):
        self.rid = rid
        self.arrival = arrival
        self.w = workload
        self.nsteps = nsteps
        self.solver = None
        self.done_steps = 0
        self.latencies_ms = []
        self.admitted_at = None
        self.finished_at = None
        self.fields = None
        self.dofs = 0


def run_serving(requests, hbm_budget_bytes, precision="fp32", keep_fields=False, max_live=64, time_scale=1.0,
                clock=time.perf_counter):
    """Serve `requests` (list of (arrival_seconds, Workload, nsteps)).  Arrival times are
    multiplied by time_scale.  Returns a dict of statistics and the finished Request objects."""
    pending = [Request(i, a * time_scale, w, n) for i, (a, w, n) in enumerate(requests)]
    pending.sort(key=lambda r: r.arrival)
    waiting, live, finished = [], [], []
    t0 = clock()
    used = 0
    ticks = 0
    max_conc = 0
    tick_ms = []
    refused_for_budget = 0
    dof_steps = 0
    while pending or waiting or live:
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.pop(0))
        # admission, oldest first, while the remaining budget allows
        still = []
        for r in waiting:
            if len(live) >= max_live:
                still.append(r)
                continue
            try:
                r.solver = Solver(r.w, precision=precision, hbm_budget_bytes=max(hbm_budget_bytes - used, 1))
            except TpnsError as e:
                if e.status == TPNS_EBUDGET:
                    refused_for_budget += 1
                    still.append(r)
                    continue
                raise
            st = r.solver.stats()
            r.dofs = st["n_fine_dofs"]
            r.bytes = st["device_bytes"]
            used += r.bytes
            r.admitted_at = clock() - t0
            live.append(r)
        waiting = still
        if not live:
            if pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - (clock() - t0))))
            continue
        max_conc = max(max_conc, len(live))
        ts = clock()
        batch_step([r.solver for r in live])
        tick_ms.append((clock() - ts) * 1e3)
        ticks += 1
        for r in live:
            r.latencies_ms.append(r.solver.stats()["last_step_ms"])
            r.done_steps += 1
            dof_steps += r.dofs
        keep = []
        for r in live:
            if r.done_steps >= r.nsteps:
                if keep_fields:
                    r.fields = r.solver.fields()
                r.solver.close()
                r.solver = None
                used -= r.bytes
                r.finished_at = clock() - t0
                finished.append(r)
            else:
                keep.append(r)
        live = keep
    wall = clock() - t0
    lat = np.array([x for r in finished for x in r.latencies_ms])
    stats = {
        "requests": len(finished), "ticks": ticks, "wall_s": wall, "max_concurrency": max_conc,
        "refused_for_budget": refused_for_budget,
        "step_latency_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
        "step_latency_ms_p99": float(np.percentile(lat, 99)) if lat.size else None,
        "tick_ms_p50": float(np.percentile(tick_ms, 50)) if tick_ms else None,
        "tick_ms_p99": float(np.percentile(tick_ms, 99)) if tick_ms else None,
        "dof_steps_per_s": dof_steps / wall if wall > 0 else None,
    }
    return stats, finished
