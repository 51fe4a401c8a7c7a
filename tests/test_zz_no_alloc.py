"""tpns_band_solve_noalloc: the band solver for callers that cannot allocate device memory
(hosts whose device memory belongs to another allocator, loops that must not allocate at
solve time).  Its scratch is a static device array inside the library.  It must return
what tpns_band_solve returns for the same system, including on consecutive calls that
reuse the array and for a system whose solve vector does not fit in shared memory."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native
    return native


def _system(native, w, j, field=0):
    import torch
    s = native.Solver(w, precision="fp64")
    s.step(1)
    info = s.debug_system(j)
    vals, rhs = s.debug_values(j, field)
    s.close()
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    return info, dev(info["rowptr"], torch.int32), dev(info["colidx"], torch.int32), dev(vals, torch.float64), \
        dev(rhs, torch.float64)


def _call(native, name, info, rp, ci, va, b, x, prec):
    lib = native.load()
    rel = C.c_double()
    fn = getattr(lib, name)
    st = fn(len(info["node"]), info["kl"], max(info["ku"], 1), C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
            C.c_void_p(va.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), native.PRECISIONS[prec],
            None, C.byref(rel))
    assert st == native.TPNS_OK, lib.tpns_last_error(None)
    return rel.value


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_solver_on_consecutive_calls(lib, prec):
    import torch
    w = W.config_small(nsteps=1)
    first = _system(lib, w, 0)            # an Oseen saddle-point system
    second = _system(lib, w, 5, field=2)  # then a Darcy system (different size and bands)
    for info, rp, ci, va, b in (first, second):
        n = len(info["node"])
        x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        x_new = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        _call(lib, "tpns_band_solve", info, rp, ci, va, b, x_ref, prec)
        rel = _call(lib, "tpns_band_solve_noalloc", info, rp, ci, va, b, x_new, prec)
        assert rel <= 1e-12
        a, r = x_new.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(a - r) <= 1e-10 * np.linalg.norm(r)


def test_noalloc_refuses_systems_beyond_its_scratch(lib):
    import torch
    lib_ = lib.load()
    n, kl = 200000, 400                   # band alone: 200000 * 801 * 4 bytes > 32 MiB
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    va = torch.zeros(1, dtype=torch.float64, device="cuda")
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = lib_.tpns_band_solve_noalloc(n, kl, kl, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
                                      C.c_void_p(va.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                      lib.PRECISIONS["fp32"], None, None)
    assert st == lib.TPNS_EINVAL
    assert b"scratch" in lib_.tpns_last_error(None)


def _banded(n, kl, ku, seed):
    """Diagonally dominant CSR matrix with bandwidths kl / ku and a right-hand side (host)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for off in range(-kl, ku + 1):
        i = np.arange(max(0, -off), min(n, n - off))
        rows.append(i)
        cols.append(i + off)
        vals.append(rng.uniform(-1.0, 1.0, len(i)) + (4.0 * (kl + ku + 1) if off == 0 else 0.0))
    r, c, v = (np.concatenate(a) for a in (rows, cols, vals))
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), v, rng.standard_normal(n)


def test_noalloc_vector_beyond_shared_memory(lib):
    """n = 30,000 in FP64 does not fit one CTA's shared memory beside a pipeline stage, so the
    solve keeps its vector in the scratch; two calls in a row match the allocating solver."""
    import torch
    n, kl, ku = 30000, 3, 2
    rp, ci, va, b = _banded(n, kl, ku, seed=11)
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    info = {"node": np.zeros(n), "kl": kl, "ku": ku}
    args = (dev(rp, torch.int32), dev(ci, torch.int32), dev(va, torch.float64), dev(b, torch.float64))
    for _ in range(2):
        x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        x_new = torch.zeros(n, dtype=torch.float64, device="cuda")
        _call(lib, "tpns_band_solve", info, *args, x_ref, "fp64")
        rel = _call(lib, "tpns_band_solve_noalloc", info, *args, x_new, "fp64")
        assert rel <= 1e-12
        a, r = x_new.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(a - r) <= 1e-10 * np.linalg.norm(r)
