"""GPU parity of the 3D configurations (Kuhn tetrahedra, P2/P1 + three P2 pressures) against
the 3D CPU oracle on the same inputs.

Tolerances (per field, relative L2 over the global fine dofs): 1e-10 for the FP64 path,
1e-8 for FP32 factors with FP64-residual refinement, as in 2D.  The steady polynomial field
is reproduced to 1e-11.  The assembled FP64 CSR values and right-hand sides of every local
system equal the oracle's to 1e-13 / 1e-12 of their scale."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme3d import TwoGridOracle3D

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-8}
FACTOR = {"mf": {}, "mf-cc": {"cuda_cores": True}, "band": {"factor": "band"}}


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as N
    N.load()
    return N


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(native, w, prec, nsteps, factor="mf"):
    o = TwoGridOracle3D(w)
    s = native.Solver(w, precision=prec, **FACTOR[factor])
    f0 = s.fields()
    for k in f0:
        assert rel(f0[k], o.fine[k]) < 1e-13, ("initial", k)
    o.run(nsteps)
    s.step(nsteps)
    f = s.fields()
    stats = s.stats()
    s.close()
    return f, o, stats


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_patch_field_exact_on_gpu_3d(native, prec):
    w = W.config_3d_patch(nsteps=2)
    f, o, _ = run_pair(native, w, prec, 2)
    ex = o.exact_fine()
    for k in f:
        assert np.abs(f[k] - ex[k]).max() < 1e-11, (k, np.abs(f[k] - ex[k]).max())


@pytest.mark.parametrize("prec,factor", [("fp64", "mf"), ("fp32", "mf"), ("fp32", "mf-cc"), ("fp64", "band"),
                                         ("fp32", "band")])
def test_small_3d_parity(native, prec, factor):
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1, nsteps=3)
    f, o, stats = run_pair(native, w, prec, 3, factor)
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))
    assert stats["last_ir_relres_max"] <= 1e-12


def test_uneven_3d_layout_parity(native):
    """Subdomains split along y and z only, overlap 2, three fine cells per coarse cell."""
    w = W.config_3d_small(n_coarse=2, r=3, nsub=(1, 2, 2), overlap=2, nsteps=2)
    f, o, _ = run_pair(native, w, "fp32", 2)
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL["fp32"], (k, rel(f[k], o.fine[k]))


def test_assembled_systems_match_oracle_3d(native):
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 1, 1), overlap=1, nsteps=1)
    o = TwoGridOracle3D(w)
    d = o.step_inputs()
    s = native.Solver(w, precision="fp64")
    s.step(1)
    nc = len(o.sub_c)
    for j in range(nc + len(o.sub_p)):
        info = s.debug_system(j)
        fields = [0] if j < nc else [0, 1, 2]
        for fld in fields:
            if j < nc:
                sub, O = o.sub_c[j]
                Aff, b, free, _ = o.local_fluid_system(j, d["t"], d["uH1h"], d["uH0h"], d["pH1h"], d["pFn_c"])
                nn = len(sub.gnode)
                key = [(int(sub.gnode[q // 3]), q % 3) if q < 3 * nn else (int(sub.gvert[q - 3 * nn]), 3) for q in free]
            else:
                sub, O = o.sub_p[j - nc]
                Aff, b, free, _ = o.local_porous_system(j - nc, fld, d["t"], d["pdH1h"], d["pdH0h"], d["ucn_p"])
                key = [(int(sub.gnode[q]), 0) for q in free]
            pos = {k: i for i, k in enumerate(key)}
            perm = np.array([pos[(int(g), int(c))] for g, c in zip(info["node"], info["comp"])])
            vals, rhs = s.debug_values(j, fld)
            A = Aff.tocsr()
            rows = np.repeat(np.arange(len(perm)), np.diff(info["rowptr"]))
            ref_vals = np.asarray(A[perm[rows], perm[info["colidx"]]]).ravel()
            assert np.abs(vals - ref_vals).max() <= 1e-13 * np.abs(ref_vals).max(), (j, fld)
            assert np.abs(rhs - b[perm]).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), (j, fld)
            assert abs(A.sum() - vals.sum()) <= 1e-12 * np.abs(A).sum()
    s.close()


def test_3d_deterministic_and_graph_equals_eager(native):
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1, nsteps=2)
    out = []
    for timing in (False, False, True):
        s = native.Solver(w, precision="fp32")
        if timing:
            s.set_timing(True)
        s.step(2)
        out.append(s.fields())
        s.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
        assert np.array_equal(out[0][k], out[2][k]), k


@pytest.mark.parametrize("dim,prec", [(2, "fp32"), (2, "fp64"), (3, "fp32"), (3, "fp64")])
def test_large_front_path_matches_one_cta_path(native, dim, prec):
    """Fronts factored by all CTAs together (forced down to order 128) give the fields of the
    one-CTA dataflow path up to the refinement's tolerance (the Schur block of a large front is
    updated once with all its pivot columns, a different rounding order), and the large-front
    path itself is deterministic."""
    w = W.config_3d_small(n_coarse=2, r=3, nsub=(1, 1, 1), overlap=1, nsteps=2) if dim == 3 else \
        W.config_graded(nsteps=2)
    out = []
    for big in (-1, 128, 128):
        s = native.Solver(w, precision=prec, mf_big_m=big)
        s.step(2)
        out.append(s.fields())
        s.close()
    for k in out[0]:
        assert rel(out[1][k], out[0][k]) <= 1e-11, (k, rel(out[1][k], out[0][k]))
        assert np.array_equal(out[1][k], out[2][k]), k


def test_large_front_path_parity_3d(native):
    w = W.config_3d_small(n_coarse=2, r=4, nsub=(1, 1, 1), overlap=1, nsteps=2)
    o = TwoGridOracle3D(w)
    o.run(2)
    s = native.Solver(w, precision="fp32", mf_big_m=256)
    s.step(2)
    f = s.fields()
    s.close()
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL["fp32"], (k, rel(f[k], o.fine[k]))
