#!/usr/bin/env python
"""Benchmark of the per-step hot path of the local parallel two-grid method (Algorithm 3,
Steps 3-4 after the coarse solve) on the 2D workload graded toward the interface:
H = 1/8, h_x = 1/128, h_y from 1/128 at Gamma to 1/32, 4 x 4 subdomains per region,
overlap 2 fine layers, log-uniform permeabilities (seed 0), dt = 0.005 -- 130,966 fine
dofs, 16 Oseen systems (3.3k-8.3k unknowns) and 48 Darcy systems per step.

Metric: fine dof-steps per second of the hot path, mixed precision (FP32 multifrontal factors
with tensor-core trailing updates, FP32 solves, FP64 assembly and refinement residuals), valid
only if every field is within relative L2 1e-8 of the FP64 GPU path on the same steps.  One
JSON line on rank 0.  The line also carries the same measurement on the 3D workload (H = 1/4,
h = 1/24, 2 x 2 x 2 subdomains per region, 721,519 fine dofs) under "workload_3d".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine DOF-steps/s at relL2<=1e-8, mixed vs FP64 GPU"
UNIT = "DOF-steps/s"
WORKLOAD = "2d_graded_H8_h128_to_h32_4x4sub_overlap2h_dt0.005 (130,966 fine dofs)"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
TF32_PER_BF16 = 0.5                                      # nominal dense TF32 / BF16 tensor rate (1.1 / 2.25)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-sample-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steps-3d", type=int, default=3,
                    help="timed steps of the 3D workload (0: skip it)")
    ap.add_argument("--serving-requests", type=int, default=16)
    ap.add_argument("--serving-steps", type=int, default=10)
    ap.add_argument("--profile", action="store_true",
                    help="only create the mixed-precision context and run W + K hot-path steps (for ncu); "
                         "prints no bench line")
    ap.add_argument("--profile-3d", action="store_true",
                    help="the same on the 3D workload (721,519 fine dofs)")
    ap.add_argument("--profile-3d-small", action="store_true",
                    help="the same on one 3D subdomain per region (H = 1/2, h = 1/12), for detailed captures")
    return ap.parse_args()


# ----------------------------------------------------------------------------- CPU oracle
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %r)
import workloads as W
from oracle.scheme import TwoGridOracle
w = W.config_graded(nsteps=%d)
o = TwoGridOracle(w)
for _ in range(%d):                       # warm-up steps
    o.step()
t0 = time.perf_counter()
for _ in range(%d):
    o.step()
dt = time.perf_counter() - t0
nd = 2 * o.mch.nn + o.mch.nv + 3 * o.mph.nn
print(json.dumps({"secs": dt, "steps": %d, "dofs": int(nd)}))
"""


def oracle_sample(nsteps, warmup=1):
    """Time the oracle (as it stands) single-threaded in a fresh process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET % (ROOT, nsteps + warmup, warmup, nsteps, nsteps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["dofs"] * d["steps"] / d["secs"], d


POOL_SNIPPET = r"""
import json, multiprocessing as mp, os, sys, time
sys.path.insert(0, %r)
import workloads as W
from oracle.scheme import TwoGridOracle

def worker(conn, mine, nsteps):
    # one rank of the paper's layout: the coarse solve (replicated) plus its own subdomains
    w = W.config_graded(nsteps=nsteps)
    o = TwoGridOracle(w)
    conn.send("ready")
    while conn.recv() == "step":
        d = o.step_inputs()
        out = {}
        for kind, j in mine:
            if kind == 0:
                out[(0, j)] = o.local_fluid(j, d["t"], d["uH1h"], d["uH0h"], d["pH1h"], d["pFn_c"])
            else:
                out[(1, j)] = o.local_porous(j, d["t"], d["pdH1h"], d["pdH0h"], d["ucn_p"])
        for (kind, j), v in out.items():
            if kind == 0:
                o.ec[j], o.dc[j] = v
            else:
                o.ep[j] = v
        o.uH, o.pH, o.pdH = d["u1"], d["p1"], d["pd1"]
        o.n += 1
        conn.send(out)

if __name__ == "__main__":
    nsteps, warm, nwork = %d, %d, %d
    w = W.config_graded(nsteps=nsteps + warm)
    o = TwoGridOracle(w)
    tasks = [(0, j) for j in range(len(o.sub_c))] + [(1, j) for j in range(len(o.sub_p))]
    nwork = max(1, min(nwork, len(tasks)))
    ctx = mp.get_context("spawn")
    pipes, procs = [], []
    for r in range(nwork):
        a, b = ctx.Pipe()
        pr = ctx.Process(target=worker, args=(b, tasks[r::nwork], nsteps + warm))
        pr.start()
        pipes.append(a)
        procs.append(pr)
    for a in pipes:
        a.recv()
    def step():
        for a in pipes:
            a.send("step")
        d = o.step_inputs()
        for a in pipes:
            for (kind, j), v in a.recv().items():
                if kind == 0:
                    o.ec[j], o.dc[j] = v
                else:
                    o.ep[j] = v
        o.uH, o.pH, o.pdH = d["u1"], d["p1"], d["pd1"]
        o.n += 1
        o.glue()
    for _ in range(warm):
        step()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        step()
    dt = time.perf_counter() - t0
    for a in pipes:
        a.send("stop")
    for pr in procs:
        pr.join()
    nd = 2 * o.mch.nn + o.mch.nv + 3 * o.mph.nn
    print(json.dumps({"secs": dt, "steps": nsteps, "dofs": int(nd), "workers": nwork}))
"""


def oracle_pool_sample(nsteps, warmup=1):
    """Time the oracle with a pool of min(#subdomains, nproc) worker processes, one per rank of
    the paper's layout (coarse solve replicated, subdomains split over the workers, glue in the
    parent), in a fresh process that starts them with spawn."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = POOL_SNIPPET % (ROOT, nsteps, warmup, os.cpu_count() or 1)
    import tempfile
    # spawned workers re-import the main module, so it has to be a file
    with tempfile.NamedTemporaryFile("w", suffix="_oracle_pool.py", delete=False) as fh:
        fh.write(code)
        path = fh.name
    try:
        r = subprocess.run([sys.executable, path], capture_output=True, text=True, env=env, timeout=1800)
    finally:
        os.unlink(path)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["dofs"] * d["steps"] / d["secs"], d


def host_cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_baseline_obj(value, d):
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['steps']} full time steps (coarse + all local solves + glue) of the same workload, "
                      f"NumPy/SciPy FP64, one thread, after warm-up steps; {d['secs']:.1f} s"}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def ndofs_of(st):
    return st["n_fine_dofs"]


def issued_tensor_flops(solver, big_m=256):
    """Tensor-core flops the FP32 factorisation of one step issues, padding included: each 32-
    column K chunk of a 128 x 128 update tile is twelve M = N = 128, K = 8 TF32 products
    (hi*hi + hi*lo + lo*hi), whatever part of the tile is inside the front.  Small fronts
    (one CTA each): after every pivot block, the whole trailing matrix in 128 x 128 tiles.
    Large fronts (order >= big_m, and their ancestors): the tile schedule of the large-front
    path (within a group of four pivot blocks, the group's own panels with one chunk; after
    the group, the trailing strips with the group's chunks; the Schur block once with all
    pivot columns).  None when the context has no multifrontal Oseen systems."""
    tile, nb, group = 128, 32, 128
    chunk = 12 * 2 * 128 * 128 * 8
    nt = lambda n: -(-n // tile) if n > 0 else 0
    total, j = 0, 0
    while True:
        info = solver.front_table(j)
        if info is None:
            break
        big = [False] * len(info)
        for t, (m, p, _lv, _par, nch, c0, c1) in enumerate(info.tolist()):
            big[t] = m >= big_m or (nch > 0 and big[c0]) or (nch > 1 and big[c1])
            for k0 in range(0, p, nb):
                k1 = min(k0 + nb, p)
                if not big[t]:
                    total += nt(m - k1) ** 2 * chunk
                    continue
                gs = (k0 // group) * group
                ge = min(gs + group, p)
                if (k0 + nb) % group:
                    if k1 < ge:
                        total += (nt(m - k1) + nt(m - ge)) * chunk
                elif ge < p:
                    b = nt(p - ge)
                    total += (nt(m - ge) * b + b * nt(m - p)) * chunk * (-(-(ge - gs) // nb))
            if big[t] and m > p:
                total += nt(m - p) ** 2 * chunk * (-(-p // nb))
        j += 1
    return total if j > 0 else None


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2311_05170_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    import workloads as W
    from paper_2311_05170_gb300.native import Solver, launch_count
    from paper_2311_05170_gb300.shard import gather_lists, max_over_ranks, shard_requests, sum_over_ranks
    K, Wm = args.steps, args.warmup
    w = W.config_graded(nsteps=Wm + K)
    stream = torch.cuda.Stream()
    handle = stream.cuda_stream
    if args.profile_3d or args.profile_3d_small:
        w3 = W.config_3d(nsteps=Wm + K) if args.profile_3d else \
            W.config_3d_small(n_coarse=2, r=6, nsub=(1, 1, 1), overlap=1, nsteps=Wm + K)
        s = Solver(w3, precision=args.precision, stream=handle)
        s.coarse_precompute(Wm + K)
        s.local_step(Wm)
        torch.cuda.synchronize()
        s.local_step(K)
        torch.cuda.synchronize()
        s.close()
        print("profile run: %d + %d hot-path steps of %s" % (Wm, K, w3.name))
        return
    if args.profile:
        s = Solver(w, precision=args.precision, stream=handle)
        s.coarse_precompute(Wm + K)
        s.local_step(Wm)
        torch.cuda.synchronize()
        s.local_step(K)
        torch.cuda.synchronize()
        s.close()
        print("profile run: %d + %d hot-path steps of %s" % (Wm, K, WORKLOAD))
        return

    def timed_hot(prec, with_phases=False, **opts):
        """K hot-path steps replayed from the captured CUDA graph (the timed region); then,
        optionally, the same number of steps launched kernel by kernel with per-phase CUDA
        events (the phase breakdown used for the roofline)."""
        s = Solver(w, precision=prec, stream=handle, **opts)
        torch.cuda.synchronize()
        tc0 = time.perf_counter()
        s.coarse_precompute(Wm + 2 * K)
        torch.cuda.synchronize()
        coarse_ms = (time.perf_counter() - tc0) * 1e3 / (Wm + 2 * K)
        s.local_step(Wm)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk = Clocks(local)
        clk.start()
        torch.cuda.synchronize()
        e0.record(stream)
        s.local_step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        launches = launch_count() - l0
        ms = max_over_ranks(ms, dist is not None, device="cuda")
        fields = s.fields()   # after Wm + K steps, before any further step
        phases = None
        if with_phases:
            # one step per call so that each step's solve passes (systems converge after
            # different numbers of refinement passes) are counted into the solve bytes
            s.set_timing(True)
            solve_bytes = 0.0
            for _ in range(K):
                s.local_step(1)
                solve_bytes += s.stats()["last_solve_bytes"]
            torch.cuda.synchronize()
            phases = s.timings()
            phases["_solve_bytes"] = solve_bytes
            s.set_timing(False)
        if phases is not None:
            phases["_coarse_ms"] = coarse_ms
        return s, ms, launches, clocks, phases, fields

    s64, ms64, _, _, _, f64 = timed_hot("fp64")
    st64 = s64.stats()
    s64.close()
    s, ms, launches, clocks, phases, f = timed_hot(args.precision, with_phases=True)
    launches = int(sum_over_ranks(launches, dist is not None, device="cuda"))   # the whole job's
    st = s.stats()
    issued = None
    if args.precision == "fp32":
        try:
            issued = issued_tensor_flops(s)
        except Exception:
            issued = None
    # both fields were read after the same Wm + K steps
    rel = {k: float(np.linalg.norm(f[k] - f64[k]) / np.linalg.norm(f64[k])) for k in f}
    # other factorisations of the local Oseen systems, same steps, error against the FP64 fields
    variants = {}
    for name, vp, opts in (("mf_fp32_cuda_cores", "fp32", {"cuda_cores": True}),
                           ("band_fp32", "fp32", {"factor": "band"}),
                           ("band_tf32_mma_sync", "tf32", {"factor": "band"}),
                           ("band_bf16_mma_sync", "bf16", {"factor": "band"}),
                           ("band_bf16_mma_sync_gmres_ir", "bf16", {"factor": "band", "gmres": True,
                                                                    "ir_classic_max": 1})):
        try:
            sv, msv, _, _, phv, fv = timed_hot(vp, with_phases=True, **opts)
            stv = sv.stats()
            sv.close()
            variants[name] = {"ms_per_step": msv / K, "value": ndofs_of(stv) * K * world / (msv / 1e3),
                              "factor_ms_per_step": phv["band_lu"][0] / K,
                              "relL2_vs_fp64_gpu_max": max(float(np.linalg.norm(fv[k] - f64[k]) / np.linalg.norm(f64[k]))
                                                           for k in fv),
                              "ir_iters_max": stv["last_ir_iters_max"], "ir_relres_max": stv["last_ir_relres_max"],
                              "gmres_cycles_last_step": stv["last_gmres_outer"], "gmres_steps": stv["gmres_steps"]}
        except Exception as ex:
            variants[name] = {"error": str(ex)[:160]}
    solve_bytes_step = phases.pop("_solve_bytes") / K
    coarse_ms = phases.pop("_coarse_ms", None)
    ph = {k: v[0] / K for k, v in phases.items()}
    phn = {k: v[1] for k, v in phases.items()}
    ndofs = st["n_fine_dofs"]
    value = ndofs * K * world / (ms / 1e3)
    value64 = ndofs * K * world / (ms64 / 1e3)
    valid = max(rel.values()) <= 1e-8
    # ---------------------------------------------------------------- roofline
    peaks = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * TF32_PER_BF16
    tsz = 4 if args.precision == "fp32" else 8
    lu_ms = ph["band_lu"]
    lu_tflops = st["band_lu_flops"] / (lu_ms / 1e3) / 1e12
    # algorithmic bytes of the HBM-bound phases (per step):
    #   Oseen assembly + scatter: CSR values 8 nnz + right-hand side 8 n + element inputs
    #     (11 FP64 geometry, 9 int32 ids, 6 nodes x 6 FP64 coarse / previous fields, 3 vertices
    #     x 2 FP64) = 88 + 36 + 288 + 48 = 460 bytes per element
    #   Darcy right-hand sides: 8 n (3 fields) + element inputs (88 + 24 + 6 x 9 x 8) = 544 B
    #   state + glue: read e_j and I_h u_H, write the glued field: 3 x 8 bytes per fine dof
    #   solves: the factor entries and block inverses of every active pass plus 24 n (see
    #     tpns_stats.last_solve_bytes), over all solve launches of a step
    asm_bytes = 8 * st["oseen_nnz"] + 8 * st["oseen_unknowns"] + 460 * st["oseen_elements"]
    darcy_bytes = 8 * st["darcy_unknowns"] + 544 * st["darcy_elements"]
    glue_bytes = 24 * ndofs

    def issued_entry(flops, ms_, peak):
        """Tensor-core flops actually issued per step and their rate over the phase time (the
        tensor pipe's busy share during the factorisation, if it ran at the TF32 peak)."""
        if not flops:
            return {}
        tf = flops / (ms_ / 1e3) / 1e12
        return {"issued_tensor_flops_per_step": flops, "issued_tflops": tf, "issued_frac_of_peak": tf / peak}

    def hbm(bytes_, ms_):
        gbs = bytes_ / (ms_ / 1e3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "ms_per_step": ms_, "bytes_per_step": bytes_}
    kernels = {
        "mf_factor": {"bound": "tensor", "achieved": lu_tflops, "peak": tf32_peak, "unit": "TFLOP/s",
                      "frac": lu_tflops / tf32_peak, "ms_per_step": lu_ms,
                      "flops_per_step": st["band_lu_flops"], "fronts": st["mf_fronts"],
                      "note": "algorithmic flops of the nested-dissection partial factorisations; the "
                              "trailing updates issue 3 TF32 products per multiply-add (split operands)",
                      **issued_entry(issued, lu_ms, tf32_peak)},
        "solves": {**hbm(solve_bytes_step, ph["solve"]), "launches_per_step": phn["solve"] / K},
        "oseen_assembly": {**hbm(asm_bytes, ph["asm_oseen"] + ph["scatter"]),
                           "limiter": "FP64 pipe (ncu: 83 % active in the element kernel; DRAM 0.6 %)"},
        "darcy_rhs": {**hbm(darcy_bytes, ph["asm_darcy"]), "limiter": "FP64 pipe (element right-hand sides in FP64)"},
        "state_glue": hbm(glue_bytes, ph["state_glue"]),
    }
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get(dom)
        except Exception:
            traffic = None
    roof = {k: v for k, v in kernels[dom].items() if k in ("bound", "achieved", "peak", "unit", "frac")}
    roof["kernel"] = dom
    roof["traffic"] = traffic
    roof["peak_source"] = ("measured bf16_tflops (MEASURED_PEAKS.json) x 1/2, the nominal TF32/BF16 ratio"
                           if roof["bound"] == "tensor" else "measured hbm_gbs (MEASURED_PEAKS.json)")
    s.close()
    # ---------------------------------------------------------------- end to end (public API, host buffers)
    torch.cuda.synchronize()
    pinned = {}
    t0 = time.perf_counter()
    e = Solver(w, precision=args.precision, stream=handle)
    torch.cuda.synchronize()
    t_created = time.perf_counter()
    d2h = 0
    for _ in range(K):
        e.step(1)
        for k in ("ux", "uy", "p", "pF", "pf", "pm"):
            if k not in pinned:
                pinned[k] = torch.empty(e.num_dofs(k), dtype=torch.float64).pin_memory()
            buf = pinned[k].numpy()
            e.field(k, out=buf)
            d2h += buf.nbytes
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    e2e_s = max_over_ranks(t_end - t0, dist is not None, device="cuda")
    steps_s = max_over_ranks(t_end - t_created, dist is not None, device="cuda")
    st_e = e.stats()
    e.close()
    e2e_val = ndofs * K * world / e2e_s
    full_ms = steps_s * 1e3 / K
    # ---------------------------------------------------------------- 3D workload
    # H = 1/4, h = 1/24, 2 x 2 x 2 subdomains per region, overlap 2 fine layers, 3D trigonometric
    # manufactured solution: 721,519 fine dofs, 8 Oseen systems of about 63k unknowns (fronts up
    # to order 3,654, 1.43e12 factorisation flops per step) and 24 Darcy systems.  Same timing
    # rules as the 2D line: W warm-up steps, K3 steps replayed from the CUDA graph on coarse
    # states precomputed in HBM, CUDA events on the library's stream; FP64 GPU path on the
    # same steps for the validity check.
    w3d = None
    if args.steps_3d > 0:
        w3 = W.config_3d(nsteps=Wm + 2 * args.steps_3d)
        K3 = args.steps_3d

        def timed_3d(prec, with_phases=False):
            s3 = Solver(w3, precision=prec, stream=handle)
            s3.coarse_precompute(Wm + 2 * K3)
            s3.local_step(Wm)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s3.local_step(K3)
            a1.record(stream)
            torch.cuda.synchronize()
            ms3 = max_over_ranks(a0.elapsed_time(a1), dist is not None, device="cuda")
            f3 = s3.fields()
            ph3 = None
            if with_phases:
                s3.set_timing(True)
                sb = 0.0
                for _ in range(K3):
                    s3.local_step(1)
                    sb += s3.stats()["last_solve_bytes"]
                torch.cuda.synchronize()
                ph3 = s3.timings()
                ph3["_solve_bytes"] = sb
                s3.set_timing(False)
            st3 = s3.stats()
            if with_phases and prec == "fp32":
                try:
                    st3["_issued"] = issued_tensor_flops(s3)
                except Exception:
                    st3["_issued"] = None
            s3.close()
            return ms3, f3, ph3, st3

        m64, g64, _, _ = timed_3d("fp64")
        m32, g32, ph3, st3 = timed_3d(args.precision, with_phases=True)
        rel3 = {k: float(np.linalg.norm(g32[k] - g64[k]) / np.linalg.norm(g64[k])) for k in g32}
        nd3 = ndofs_of(st3)
        v3 = nd3 * K3 * world / (m32 / 1e3)
        v64 = nd3 * K3 * world / (m64 / 1e3)
        p3 = {k: v[0] / K3 for k, v in ph3.items() if not k.startswith("_")}
        f_ms = p3["band_lu"]
        f_tf = st3["band_lu_flops"] / (f_ms / 1e3) / 1e12
        sb3 = ph3["_solve_bytes"] / K3
        w3d = {
            "workload": "3d_H4_h24_2x2x2sub_overlap2h_dt0.01 (%s fine dofs)" % format(nd3, ","),
            "value": v3 if max(rel3.values()) <= 1e-8 else None, "unit": UNIT, "ms_per_step": m32 / K3,
            "steps": K3, "warmup": Wm, "valid": max(rel3.values()) <= 1e-8, "relL2_vs_fp64_gpu": rel3,
            "fp64_gpu": {"value": v64, "ms_per_step": m64 / K3}, "speedup_vs_fp64_gpu": v3 / v64,
            "phases_ms_per_step": p3,
            "mf_factor": {"bound": "tensor", "achieved": f_tf, "peak": tf32_peak, "unit": "TFLOP/s",
                          "frac": f_tf / tf32_peak, "ms_per_step": f_ms, "flops_per_step": st3["band_lu_flops"],
                          "fronts": st3["mf_fronts"],
                          "note": "fronts of order >= 256 and their ancestors factored by all CTAs per tree level",
                          **issued_entry(st3.get("_issued"), f_ms, tf32_peak)},
            "solves": {**hbm(sb3, p3["solve"])},
            "ir": {"iters_max": st3["last_ir_iters_max"], "relres_max": st3["last_ir_relres_max"]},
            "config": {"oseen_unknowns": st3["oseen_unknowns"], "oseen_nnz": st3["oseen_nnz"],
                       "oseen_elements": st3["oseen_elements"], "factor_entries": st3["factor_entries"],
                       "device_bytes": st3["device_bytes"], "create_ms": st3["create_ms"],
                       "l2": "inputs larger than L2 (fronts %.1f GB)" % (st3["factor_entries"] * tsz / 1e9)},
        }
    # ---------------------------------------------------------------- serving (bounded sample)
    serving = None
    if args.serving_requests > 0:
        # each rank serves its own share of the requests (no collective while serving)
        from paper_2311_05170_gb300.serve import run_serving
        reqs = [(a, rw, args.serving_steps) for a, rw in W.serving_requests()[: args.serving_requests]]
        mine = shard_requests(reqs, rank, world)
        sstats, done = run_serving(mine, hbm_budget_bytes=64 << 30, precision=args.precision)
        on = dist is not None
        lat = np.array(gather_lists([x for r in done for x in r.latencies_ms], on))
        obs = np.array(gather_lists([x for r in done for x in r.observed_ms], on))
        wall = max_over_ranks(sstats["wall_s"], on, device="cuda")
        serving = {
            "requests": int(sum_over_ranks(sstats["requests"], on, device="cuda")),
            "ticks_max": int(max_over_ranks(sstats["ticks"], on, device="cuda")),
            "wall_s": wall,
            "max_concurrency_per_gpu": int(max_over_ranks(sstats["max_concurrency"], on, device="cuda")),
            "refused_for_budget": int(sum_over_ranks(sstats["refused_for_budget"], on, device="cuda")),
            "step_latency_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
            "step_latency_ms_p99": float(np.percentile(lat, 99)) if lat.size else None,
            "observed_step_latency_ms_p50": float(np.percentile(obs, 50)) if obs.size else None,
            "observed_step_latency_ms_p99": float(np.percentile(obs, 99)) if obs.size else None,
            "tick_ms_max_p50": max_over_ranks(sstats["tick_ms_p50"] or 0.0, on, device="cuda"),
            "dof_steps_per_s": sum_over_ranks(sum(r.dofs * r.done_steps for r in done), on, device="cuda") / wall,
            "sample": (f"first {args.serving_requests} of the 512 seeded requests (Poisson arrivals, 20/s), "
                       f"{args.serving_steps} steps each, sharded over {world} GPU(s) by estimated work, "
                       f"HBM budget 64 GiB per GPU; step latency = device time of a request's step within "
                       f"its batched tick (other requests running beside it); observed step latency = wall time "
                       f"from the step's readiness (end of the request's previous step, or its admission) to "
                       f"the end of its tick; contexts created by a background thread beside the ticks; wall "
                       f"includes context creation"),
        }
    # ---------------------------------------------------------------- CPU baseline (oracle)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            v, d = oracle_sample(args.cpu_sample_steps)
            cpu = cpu_baseline_obj(v, d)
        except Exception as ex:  # the line still reports the GPU numbers
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
        cpu["nproc"] = os.cpu_count()
        cpu["cpu_model"] = host_cpu_model()
        try:
            vp, dp = oracle_pool_sample(args.cpu_sample_steps)
            cpu["pool"] = {"value": vp, "unit": UNIT, "cores": dp["workers"],
                           "sample": f"{dp['steps']} full time steps, {dp['workers']} worker processes (spawned): "
                                     "the coarse solve replicated in every worker, the 32 subdomain problems "
                                     "split over the workers, the glue in the parent; "
                                     f"{dp['secs']:.1f} s"}
        except Exception as ex:
            cpu["pool"] = {"value": None, "sample": f"failed: {str(ex)[:200]}"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value if valid else None, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fine_dofs": ndofs, "local_systems_per_step": st["n_local_systems"],
                       "replicas": world, "l2": "inputs larger than L2 (multifrontal fronts %.0f MB per replica)"
                       % (st["factor_entries"] * tsz / 1e6),
                       "parallelism": "independent replicas (no data-path collective)",
                       "factorisation": "multifrontal (nested dissection), FP32 fronts, tcgen05 split-TF32 "
                                        "trailing updates",
                       "timed": "K hot-path steps (prolongation, assembly, multifrontal LU, solves + FP64 "
                                "refinement, glue) replayed from a CUDA graph on coarse states precomputed in HBM; "
                                "per-phase times from K further steps launched kernel by kernel"},
            "valid": valid, "relL2_vs_fp64_gpu": rel,
            "fp64_gpu": {"value": value64, "ms_per_step": ms64 / K},
            "factorisation_variants": {
                "what": "other factorisations of the local Oseen systems on the same steps: the multifrontal "
                        "LU with CUDA-core trailing updates, and the band LU (FP32 FMA; mma.sync TF32 with "
                        "split operands; mma.sync plain BF16, with classic refinement and with one classic "
                        "pass followed by GMRES-based refinement); FP64-residual refinement throughout",
                **variants},
            "speedup_vs_fp64_gpu": value / value64,
            "roofline": roof, "kernels": kernels,
            "phases_ms_per_step": ph,
            "ir": {"iters_max": st["last_ir_iters_max"], "relres_max": st["last_ir_relres_max"]},
            "coarse_solve": {"ms_per_step": coarse_ms,
                             "what": "Step 1 alone (coarse Darcy solves with the factors kept from create, "
                                     "Newton Navier-Stokes with FP32 factors refined against the FP64 "
                                     "Jacobian) on the GPU: wall time of the coarse trajectory the timed "
                                     "steps read, over its steps; not part of the hot-path value"},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": st_e["h2d_bytes"] / K,
                    "d2h_bytes_per_step": d2h / K,
                    "what": "tpns_create from host descriptors (its uploads amortised over the K steps) + K x "
                            "(tpns_step incl. the coarse solve + tpns_get_field of all 6 fields into pinned host "
                            "memory)",
                    "create_ms": (t_created - t0) * 1e3, "create_ms_library": st_e["create_ms"],
                    "full_step_ms": full_ms,
                    "full_step_what": "one tpns_step (coarse solve + hot path) plus the read-back of all fields, "
                                      "create excluded"},
            "gpu_launches": launches,
            "workload_3d": w3d,
            "serving": serving,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args, rank):
    """The oracle as the reference implementation, timed on the host cores."""
    if rank != 0:
        return
    v, d = oracle_sample(args.steps, warmup=args.warmup)
    cpu = cpu_baseline_obj(v, d)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": d["secs"] * 1e3 / d["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fine_dofs": 130966, "local_systems_per_step": 64, "replicas": 1,
                       "parallelism": "oracle on the host cores (one thread)",
                       "timed": "full time steps of the oracle (coarse solve, all local solves, glue)"},
            "impl": "reference", "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
