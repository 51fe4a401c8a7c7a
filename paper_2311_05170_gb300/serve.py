"""Serving loop for many simulations of the two-grid method on one GPU (continuous batching).

Requests arrive over time (Poisson arrivals); each is a simulation with its own mesh sizes and
physical parameters.  A request is admitted when the device memory it needs fits in the HBM
budget left by the simulations on the device (the library refuses a context whose footprint
exceeds the budget it is given: TPNS_EBUDGET); its coarse and fine state and its Darcy factors
then stay resident until it has run its steps.  Contexts are created by a background thread,
on streams that do not synchronise with the legacy default stream, so admitting a request
overlaps with the steps of the simulations already running.  Every scheduler tick advances all
admitted simulations by one time step with one tpns_batch_step call: their steps are enqueued
side by side on their own streams, so their work overlaps on the device.  Finished simulations
are released at once, which frees memory for waiting ones.

Two per-step latencies are recorded for every request step:
  * device: the device time of the step within its tick, from the step's start on the
    simulation's stream to its end, with the other simulations running beside it
    (tpns_stats.last_step_ms);
  * observed: wall time from the moment the step could start (the end of the request's previous
    step, or its admission) to the end of the tick that carried it -- what a client waiting for
    each step sees, including the wait for the slowest simulation of the tick.
"""
import threading
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
        self.stream = None
        self.done_steps = 0
        self.latencies_ms = []
        self.observed_ms = []
        self.admitted_at = None
        self.ready_at = None
        self.finished_at = None
        self.fields = None
        self.dofs = 0
        self.bytes = 0


def _stream():
    """A CUDA stream that does not synchronise with the legacy default stream (None if torch
    is not available: the library then creates its own stream)."""
    try:
        import torch
        return torch.cuda.Stream()
    except Exception:
        return None


def run_serving(requests, hbm_budget_bytes, precision="fp32", keep_fields=False, max_live=64, time_scale=1.0,
                clock=time.perf_counter, background=True):
    """Serve `requests` (list of (arrival_seconds, Workload, nsteps)).  Arrival times are
    multiplied by time_scale.  background=False creates the contexts in the scheduler loop itself
    between ticks (a deterministic schedule, used to test the policy).  Returns a dict of
    statistics and the finished Request objects."""
    pending = [Request(i, a * time_scale, w, n) for i, (a, w, n) in enumerate(requests)]
    pending.sort(key=lambda r: r.arrival)
    lock = threading.Lock()
    state = {"used": 0, "refused": 0, "error": None, "stop": False, "live": 0, "changed": 0}
    waiting, ready = [], []
    t0 = clock()

    def admit_one():
        """Try the waiting requests oldest first; create the first one that fits the budget
        left.  Returns True if one was admitted."""
        with lock:
            snapshot = list(waiting)
            room = max_live - state["live"] - len(ready)
        if room <= 0:
            return False
        for r in snapshot:
            with lock:
                left = hbm_budget_bytes - state["used"]
            try:
                r.stream = _stream()
                handle = r.stream.cuda_stream if r.stream is not None else None
                solver = Solver(r.w, precision=precision, hbm_budget_bytes=max(left, 1), stream=handle)
            except TpnsError as e:
                if e.status == TPNS_EBUDGET:
                    with lock:
                        state["refused"] += 1
                    continue
                raise
            st = solver.stats()
            with lock:
                r.solver = solver
                r.dofs = st["n_fine_dofs"]
                r.bytes = st["device_bytes"]
                state["used"] += r.bytes
                r.admitted_at = clock() - t0
                r.ready_at = r.admitted_at
                waiting.remove(r)
                ready.append(r)
            return True
        return False

    def creator():
        seen = -1
        while not state["stop"]:
            with lock:
                changed = state["changed"]
                nwait = len(waiting)
            if nwait == 0 or changed == seen:
                time.sleep(0.0005)
                continue
            try:
                if not admit_one():
                    seen = changed        # nothing fits until a simulation finishes or a request arrives
            except Exception as e:       # noqa: BLE001 - reported to the caller
                state["error"] = e
                return

    th = None
    if background:
        th = threading.Thread(target=creator, daemon=True)
        th.start()
    live, finished = [], []
    idle_since = clock()
    ticks = 0
    max_conc = 0
    tick_ms = []
    dof_steps = 0
    try:
        while pending or waiting or live or ready:
            if state["error"] is not None:
                raise state["error"]
            now = clock() - t0
            with lock:
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.pop(0))
                    state["changed"] += 1
            if not background:
                while admit_one():
                    pass
            with lock:
                live.extend(ready)
                ready.clear()
                state["live"] = len(live)
            if not live:
                with lock:
                    stuck = waiting and not pending and not ready
                if stuck and (not background or clock() - idle_since > 30.0):
                    raise RuntimeError("a request does not fit the HBM budget on an empty device")
                time.sleep(0.0005)
                continue
            idle_since = clock()
            max_conc = max(max_conc, len(live))
            ts = clock()
            batch_step([r.solver for r in live])
            te = clock()
            tick_ms.append((te - ts) * 1e3)
            ticks += 1
            for r in live:
                r.latencies_ms.append(r.solver.stats()["last_step_ms"])
                r.observed_ms.append((te - t0 - r.ready_at) * 1e3)
                r.ready_at = te - t0
                r.done_steps += 1
                dof_steps += r.dofs
            keep = []
            for r in live:
                if r.done_steps >= r.nsteps:
                    if keep_fields:
                        r.fields = r.solver.fields()
                    r.solver.close()
                    r.solver = None
                    with lock:
                        state["used"] -= r.bytes
                        state["changed"] += 1
                    r.finished_at = clock() - t0
                    finished.append(r)
                else:
                    keep.append(r)
            live = keep
            with lock:
                state["live"] = len(live)
    finally:
        state["stop"] = True
        if th is not None:
            th.join(timeout=30)
    wall = clock() - t0
    lat = np.array([x for r in finished for x in r.latencies_ms])
    obs = np.array([x for r in finished for x in r.observed_ms])
    stats = {
        "requests": len(finished), "ticks": ticks, "wall_s": wall, "max_concurrency": max_conc,
        "refused_for_budget": state["refused"],
        "step_latency_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
        "step_latency_ms_p99": float(np.percentile(lat, 99)) if lat.size else None,
        "observed_step_latency_ms_p50": float(np.percentile(obs, 50)) if obs.size else None,
        "observed_step_latency_ms_p99": float(np.percentile(obs, 99)) if obs.size else None,
        "tick_ms_p50": float(np.percentile(tick_ms, 50)) if tick_ms else None,
        "tick_ms_p99": float(np.percentile(tick_ms, 99)) if tick_ms else None,
        "dof_steps_per_s": dof_steps / wall if wall > 0 else None,
    }
    return stats, finished
