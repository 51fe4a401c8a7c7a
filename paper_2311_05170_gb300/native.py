"""ctypes binding of the C ABI declared in include/tpns.h (argument marshalling only).

Every computation runs in libtpns.so; this module raises if the library is missing."""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtpns.so")

TPNS_OK, TPNS_EINVAL, TPNS_ENOMEM, TPNS_ENOTCONV, TPNS_EDEVICE, TPNS_ETIMEOUT, TPNS_EBUDGET, TPNS_EBREAKDOWN = range(8)
STATUS_NAMES = ["TPNS_OK", "TPNS_EINVAL", "TPNS_ENOMEM", "TPNS_ENOTCONV", "TPNS_EDEVICE", "TPNS_ETIMEOUT",
                "TPNS_EBUDGET", "TPNS_EBREAKDOWN"]
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
MAX_COARSE_ROWS = 64


class MeshDesc(C.Structure):
    _fields_ = [("nx_coarse", C.c_int32), ("ny_coarse", C.c_int32), ("fine_per_coarse_x", C.c_int32),
                ("fine_rows_from_gamma", C.c_int32 * MAX_COARSE_ROWS), ("dim", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("nu", C.c_double), ("eta", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("alpha", C.c_double), ("sigma", C.c_double), ("sigma_star", C.c_double),
                ("phiC", C.c_double * 3), ("k", C.c_double * 3)]


class PartitionDesc(C.Structure):
    _fields_ = [("nsub_x", C.c_int32), ("nsub_y", C.c_int32), ("overlap", C.c_int32), ("nsub_z", C.c_int32)]


class DataDesc(C.Structure):
    _fields_ = [("mms_id", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("local_factor", C.c_int32), ("mf_leaf", C.c_int32), ("mf_cuda_cores", C.c_int32),
                ("mf_ctas", C.c_int32), ("rank", C.c_int32), ("nranks", C.c_int32), ("algorithm", C.c_int32),
                ("refinement", C.c_int32), ("ir_classic_max", C.c_int32), ("mf_big_m", C.c_int32)]


FACTORS = {"mf": 0, "band": 1}


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("last_ir_iters_max", C.c_int32), ("last_newton_iters", C.c_int32),
                ("last_ir_relres_max", C.c_double), ("n_fine_dofs", C.c_int64), ("n_local_systems", C.c_int64),
                ("device_bytes", C.c_int64), ("band_lu_flops", C.c_double), ("h2d_bytes", C.c_int64),
                ("last_ir_solves", C.c_int64), ("last_solve_bytes", C.c_double), ("last_step_ms", C.c_double),
                ("lu_cluster_ctas", C.c_int64), ("oseen_unknowns", C.c_int64), ("oseen_nnz", C.c_int64),
                ("oseen_elements", C.c_int64), ("darcy_unknowns", C.c_int64), ("darcy_elements", C.c_int64),
                ("factor_entries", C.c_double), ("mf_fronts", C.c_int64), ("create_ms", C.c_double),
                ("last_gmres_outer", C.c_int32), ("gmres_steps", C.c_int32)]


class TpnsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None

EXPORTS = ["tpns_create", "tpns_step", "tpns_coarse_precompute", "tpns_local_step", "tpns_num_dofs",
           "tpns_get_field", "tpns_get_stats", "tpns_batch_step", "tpns_last_error", "tpns_destroy",
           "tpns_debug_mesh", "tpns_debug_system", "tpns_set_timing", "tpns_get_timings", "tpns_launch_count",
           "tpns_layout_create", "tpns_debug_values", "tpns_band_solve",
           "tpns_band_solve_noalloc", "tpns_create_ex", "tpns_layout_create_ex", "tpns_debug_fronts"]

PHASES = ["coarse", "prolong", "asm_oseen", "scatter", "asm_darcy", "band_fill", "band_lu", "solve", "residual",
          "state_glue", "copies"]


def load(path=LIB_PATH):
    """Load libtpns.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libtpns.so not found at {path}; build it with paper_2311_05170_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.tpns_create.argtypes = [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(PartitionDesc),
                                C.POINTER(DataDesc), C.c_double, C.c_int, C.c_size_t, P, C.POINTER(P)]
    lib.tpns_create.restype = C.c_int
    lib.tpns_create_ex.argtypes = [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(PartitionDesc),
                                   C.POINTER(DataDesc), C.c_double, C.c_int, C.c_size_t, P, C.POINTER(Options),
                                   C.POINTER(P)]
    lib.tpns_create_ex.restype = C.c_int
    lib.tpns_layout_create_ex.argtypes = [C.POINTER(MeshDesc), C.POINTER(PartitionDesc), C.POINTER(Options),
                                          C.POINTER(P)]
    lib.tpns_layout_create_ex.restype = C.c_int
    lib.tpns_debug_fronts.argtypes = [P, C.c_int32, C.c_int32, P, C.POINTER(C.c_size_t)]
    lib.tpns_debug_fronts.restype = C.c_int
    for name in ("tpns_step", "tpns_coarse_precompute", "tpns_local_step"):
        getattr(lib, name).argtypes = [P, C.c_int32]
        getattr(lib, name).restype = C.c_int
    lib.tpns_num_dofs.argtypes = [P, C.c_int32, C.POINTER(C.c_size_t)]
    lib.tpns_num_dofs.restype = C.c_int
    lib.tpns_get_field.argtypes = [P, C.c_int32, P, C.c_size_t, C.c_int32]
    lib.tpns_get_field.restype = C.c_int
    lib.tpns_get_stats.argtypes = [P, C.POINTER(Stats)]
    lib.tpns_get_stats.restype = C.c_int
    lib.tpns_batch_step.argtypes = [C.POINTER(P), C.c_int32]
    lib.tpns_batch_step.restype = C.c_int
    lib.tpns_last_error.argtypes = [P]
    lib.tpns_last_error.restype = C.c_char_p
    lib.tpns_destroy.argtypes = [P]
    lib.tpns_destroy.restype = None
    lib.tpns_debug_mesh.argtypes = [P, C.c_int32, P, C.POINTER(C.c_size_t)]
    lib.tpns_debug_mesh.restype = C.c_int
    I32 = C.POINTER(C.c_int32)
    lib.tpns_debug_system.argtypes = [P, C.c_int32, I32, I32, I32, C.POINTER(C.c_int64), I32, I32, I32, I32]
    lib.tpns_debug_system.restype = C.c_int
    lib.tpns_set_timing.argtypes = [P, C.c_int32]
    lib.tpns_set_timing.restype = C.c_int
    lib.tpns_get_timings.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]
    lib.tpns_get_timings.restype = C.c_int
    lib.tpns_launch_count.argtypes = []
    lib.tpns_launch_count.restype = C.c_int64
    lib.tpns_layout_create.argtypes = [C.POINTER(MeshDesc), C.POINTER(PartitionDesc), C.POINTER(P)]
    lib.tpns_layout_create.restype = C.c_int
    lib.tpns_debug_values.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.tpns_debug_values.restype = C.c_int
    lib.tpns_band_solve.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, C.c_int, P,
                                    C.POINTER(C.c_double)]
    lib.tpns_band_solve.restype = C.c_int
    lib.tpns_band_solve_noalloc.argtypes = lib.tpns_band_solve.argtypes
    lib.tpns_band_solve_noalloc.restype = C.c_int
    _lib = lib
    return lib


def _check(lib, ctx, status):
    if status != TPNS_OK:
        msg = lib.tpns_last_error(ctx)
        raise TpnsError(status, msg.decode() if msg else "")


def descriptors(w):
    """ABI descriptors of a workloads.Workload."""
    md = MeshDesc()
    p = w.params
    pr = Params(p.nu, p.eta, p.rho, p.mu, p.alpha, p.sigma, p.sigma_star, (C.c_double * 3)(*p.phiC),
                (C.c_double * 3)(*p.k))
    if getattr(w, "dim", 2) == 3:
        md.nx_coarse = md.ny_coarse = w.n_coarse
        md.fine_per_coarse_x = w.fine_per_coarse
        md.dim = 3
        pd = PartitionDesc(w.nsub[0], w.nsub[1], w.overlap, w.nsub[2])
        return md, pr, pd, DataDesc(w.mms)
    md.nx_coarse, md.ny_coarse, md.fine_per_coarse_x = w.nx_coarse, w.ny_coarse, w.fine_per_coarse_x
    for c, m in enumerate(w.fine_rows_from_gamma):
        md.fine_rows_from_gamma[c] = m
    md.dim = 2
    pd = PartitionDesc(w.nsub[0], w.nsub[1], w.overlap, 1)
    dd = DataDesc(w.mms)
    return md, pr, pd, dd


FIELD_IDS = {"ux": 0, "uy": 1, "p": 2, "pF": 3, "pf": 4, "pm": 5}
FIELD_IDS_3D = {"ux": 0, "uy": 1, "uz": 2, "p": 3, "pF": 4, "pf": 5, "pm": 6}


class Solver:
    """One simulation context on the current CUDA device (host_only=True: layout only)."""

    def __init__(self, w, precision="fp64", hbm_budget_bytes=0, stream=None, host_only=False, factor="mf",
                 mf_leaf=0, cuda_cores=False, mf_ctas=0, rank=0, nranks=0, algorithm=3, gmres=False,
                 ir_classic_max=0, mf_big_m=0):
        self.lib = load()
        self.w = w
        self.ids = FIELD_IDS_3D if getattr(w, "dim", 2) == 3 else FIELD_IDS
        md, pr, pd, dd = descriptors(w)
        opt = Options(FACTORS[factor], int(mf_leaf), 1 if cuda_cores else 0, int(mf_ctas), int(rank), int(nranks),
                      int(algorithm), 1 if gmres else 0, int(ir_classic_max), int(mf_big_m))
        ctx = C.c_void_p()
        if host_only:
            _check(self.lib, None, self.lib.tpns_layout_create_ex(C.byref(md), C.byref(pd), C.byref(opt),
                                                                  C.byref(ctx)))
            self.ctx = ctx
            return
        st = C.c_void_p(stream) if stream else None
        s = self.lib.tpns_create_ex(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), float(w.dt),
                                    PRECISIONS[precision], int(hbm_budget_bytes), st, C.byref(opt), C.byref(ctx))
        _check(self.lib, None, s)
        self.ctx = ctx

    def step(self, n=1):
        _check(self.lib, self.ctx, self.lib.tpns_step(self.ctx, int(n)))

    def coarse_precompute(self, n):
        _check(self.lib, self.ctx, self.lib.tpns_coarse_precompute(self.ctx, int(n)))

    def local_step(self, n=1):
        _check(self.lib, self.ctx, self.lib.tpns_local_step(self.ctx, int(n)))

    def num_dofs(self, field):
        n = C.c_size_t()
        _check(self.lib, self.ctx, self.lib.tpns_num_dofs(self.ctx, self.ids.get(field, field), C.byref(n)))
        return n.value

    def field(self, field, out=None):
        """Glued global fine field as a NumPy array (host copy)."""
        fid = self.ids.get(field, field)
        n = self.num_dofs(fid)
        if out is None:
            out = np.empty(n, dtype=np.float64)
        _check(self.lib, self.ctx, self.lib.tpns_get_field(self.ctx, fid, out.ctypes.data, n, 0))
        return out

    def field_to_device(self, field, dev_ptr, n):
        fid = self.ids.get(field, field)
        _check(self.lib, self.ctx, self.lib.tpns_get_field(self.ctx, fid, C.c_void_p(dev_ptr), n, 1))

    def fields(self):
        return {k: self.field(k) for k in self.ids}

    def stats(self):
        s = Stats()
        _check(self.lib, self.ctx, self.lib.tpns_get_stats(self.ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def debug_mesh(self, what):
        n = C.c_size_t()
        _check(self.lib, self.ctx, self.lib.tpns_debug_mesh(self.ctx, what, None, C.byref(n)))
        out = np.empty(n.value, dtype=np.float64 if what in (0, 1) else np.int32)
        _check(self.lib, self.ctx, self.lib.tpns_debug_mesh(self.ctx, what, out.ctypes.data, C.byref(n)))
        return out

    def debug_system(self, j):
        lib = self.lib
        n = C.c_int32()
        nnz = C.c_int64()
        kl, ku = C.c_int32(), C.c_int32()
        _check(lib, self.ctx, lib.tpns_debug_system(self.ctx, j, C.byref(n), None, None, C.byref(nnz), None, None,
                                                    C.byref(kl), C.byref(ku)))
        node = np.empty(n.value, np.int32)
        comp = np.empty(n.value, np.int32)
        rp = np.empty(n.value + 1, np.int32)
        ci = np.empty(nnz.value, np.int32)
        I32 = C.POINTER(C.c_int32)
        _check(lib, self.ctx, lib.tpns_debug_system(self.ctx, j, None, node.ctypes.data_as(I32),
                                                    comp.ctypes.data_as(I32), None, rp.ctypes.data_as(I32),
                                                    ci.ctypes.data_as(I32), None, None))
        return {"node": node, "comp": comp, "rowptr": rp, "colidx": ci, "kl": kl.value, "ku": ku.value}

    def front_table(self, j):
        """Per front of local Oseen system j (children before parents): m, p, level, parent,
        nchild, child0, child1 (tpns_debug_fronts, what = 1); None when j is not an Oseen
        system of a multifrontal context."""
        lib = self.lib
        n = C.c_size_t()
        if lib.tpns_debug_fronts(self.ctx, int(j), 1, None, C.byref(n)) != 0:
            return None
        out = np.empty(n.value, np.int32)
        _check(lib, self.ctx, lib.tpns_debug_fronts(self.ctx, int(j), 1, out.ctypes.data, C.byref(n)))
        return out.reshape(-1, 7)

    def debug_fronts(self, j):
        """Multifrontal structure of local Oseen system j (see tpns_debug_fronts)."""
        lib = self.lib

        def get(what):
            n = C.c_size_t()
            _check(lib, self.ctx, lib.tpns_debug_fronts(self.ctx, j, what, None, C.byref(n)))
            out = np.empty(n.value, np.int32)
            _check(lib, self.ctx, lib.tpns_debug_fronts(self.ctx, j, what, out.ctypes.data, C.byref(n)))
            return out

        nf, nlev = get(0)
        info = get(1).reshape(nf, 7)
        fronts = []
        rows, rel, cp, ok, oi, cc = get(2), get(3), get(4), get(5), get(6), get(7)
        a = b = c = d = 0
        for t in range(nf):
            m, p = int(info[t, 0]), int(info[t, 1])
            cptr = cp[c:c + m + 1].copy()
            fronts.append({"m": m, "p": p, "level": int(info[t, 2]), "parent": int(info[t, 3]),
                           "children": [int(x) for x in info[t, 5:5 + info[t, 4]]], "rows": rows[a:a + m].copy(),
                           "relmap": rel[b:b + m - p].copy() if info[t, 3] >= 0 else np.empty(0, np.int32),
                           "col_ptr": cptr, "orig_k": ok[d:d + cptr[-1]].copy(), "orig_i": oi[d:d + cptr[-1]].copy(),
                           "col_child": cc[2 * a:2 * a + 2 * m].reshape(m, 2).copy()})
            a += m
            b += m - p if info[t, 3] >= 0 else 0
            c += m + 1
            d += cptr[-1]
        return {"nlevels": int(nlev), "fronts": fronts, "order": get(8)}

    def set_timing(self, on=True):
        _check(self.lib, self.ctx, self.lib.tpns_set_timing(self.ctx, 1 if on else 0))

    def timings(self):
        """Per-phase totals {phase: (ms, intervals)} measured with CUDA events."""
        n = len(PHASES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        _check(self.lib, self.ctx, self.lib.tpns_get_timings(self.ctx, ms, cnt, n))
        return {PHASES[i]: (ms[i], cnt[i]) for i in range(n)}

    def debug_values(self, j, field=0):
        info = self.debug_system(j)
        vals = np.empty(len(info["colidx"]), np.float64)
        rhs = np.empty(len(info["node"]), np.float64)
        _check(self.lib, self.ctx, self.lib.tpns_debug_values(self.ctx, j, field, vals.ctypes.data, rhs.ctypes.data))
        return vals, rhs

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tpns_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def band_solve(n, kl, ku, rowptr, colidx, vals, b, x, precision="fp32", stream=None):
    """Solve A x = b with device pointers (int addresses); returns the final relative
    residual.  See tpns_band_solve in include/tpns.h."""
    lib = load()
    rel = C.c_double()
    st = lib.tpns_band_solve(int(n), int(kl), int(ku), C.c_void_p(rowptr), C.c_void_p(colidx), C.c_void_p(vals),
                             C.c_void_p(b), C.c_void_p(x), PRECISIONS[precision],
                             C.c_void_p(stream) if stream else None, C.byref(rel))
    _check(lib, None, st)
    return rel.value


def launch_count():
    return load().tpns_launch_count()


def batch_step(solvers):
    lib = load()
    arr = (C.c_void_p * len(solvers))(*[s.ctx for s in solvers])
    _check(lib, None, lib.tpns_batch_step(arr, len(solvers)))
