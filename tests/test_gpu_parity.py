"""GPU parity of the native library against the CPU oracle (same seeded inputs).

Tolerances (per field, relative L2 over the global fine dofs): 1e-10 for the FP64 path,
1e-8 for FP32 factors with FP64-residual refinement.  Both sides integrate the
transcendental data with the same quadrature rules, so the only differences are rounding
orders and the refinement's stopping point.  The local Oseen systems are factored by the
multifrontal LU (default: tensor-core trailing updates for FP32 fronts; "mf-cc": CUDA-core
updates) or by the band LU ("band")."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme import TwoGridOracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-8, "tf32": 1e-8, "bf16": 1e-8}


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


FACTOR = {"mf": {}, "mf-cc": {"cuda_cores": True}, "band": {"factor": "band"}}


def run_pair(native, w, prec, nsteps, factor="mf"):
    o = TwoGridOracle(w)
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
@pytest.mark.parametrize("factor", ["mf", "band"])
def test_patch_field_exact_on_gpu(native, prec, factor):
    w = W.config_patch(nx_coarse=2, r=2, nsub=(2, 2), nsteps=3)
    f, o, _ = run_pair(native, w, prec, 3, factor)
    ex = o.exact_fine()
    for k in f:
        assert np.abs(f[k] - ex[k]).max() < 1e-11, k


@pytest.mark.parametrize("prec,factor", [("fp64", "mf"), ("fp32", "mf"), ("fp32", "mf-cc"), ("tf32", "mf"),
                                         ("fp64", "band"), ("fp32", "band"), ("tf32", "band"), ("bf16", "band")])
def test_small_2d_parity(native, prec, factor):
    w = W.config_small(nsteps=10)
    f, o, stats = run_pair(native, w, prec, 10, factor)
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))
    assert stats["last_ir_relres_max"] <= 1e-12


@pytest.mark.parametrize("prec,factor", [("fp64", "mf"), ("fp32", "mf"), ("fp32", "mf-cc"), ("fp32", "band"),
                                         ("tf32", "band")])
def test_graded_full_size_parity(native, prec, factor):
    """The bench workload at full size (130,966 fine dofs, 16 + 48 local systems of 1.4k to
    8.3k unknowns), three steps."""
    w = W.config_graded(nsteps=3)
    f, o, stats = run_pair(native, w, prec, 3, factor)
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))
    assert stats["n_fine_dofs"] == 130966 and stats["n_local_systems"] == 64


@pytest.mark.parametrize("w", [W.config_uniform(4, 2, nsub=(1, 1), overlap=1, nsteps=3),
                               W.config_uniform(8, 2, nsub=(4, 2), overlap=3, nsteps=3),
                               W.config_uniform(4, 1, nsub=(2, 2), overlap=1, nsteps=3)],
                         ids=["single_subdomain", "uneven_4x2", "H_equals_h"])
@pytest.mark.parametrize("factor", ["mf", "band"])
def test_edge_layouts_parity(native, w, factor):
    f, o, _ = run_pair(native, w, "fp32", 3, factor)
    for k in f:
        assert rel(f[k], o.fine[k]) <= 1e-8, k


def test_wide_band_parity(native):
    """Subdomains whose Oseen band (kl = 851) is taller than the LU CTA has threads: the panel
    is factored from shared memory and the solve vector lives in global scratch; FP32 with
    FP64 refinement still meets the mixed-precision tolerance against the oracle."""
    w = W.config_uniform(4, 24, nsub=(2, 2), nsteps=2)
    s = native.Solver(w, precision="fp32", host_only=True)
    assert max(s.debug_system(j)["kl"] for j in range(4)) == 851
    s.close()
    f, o, stats = run_pair(native, w, "fp32", 2, "band")
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL["fp32"], (k, rel(f[k], o.fine[k]))
    assert stats["last_ir_relres_max"] <= 1e-12


def test_widest_band_global_vector_parity(native):
    """h = 1/128 with 2 x 2 subdomains per region: Oseen bands of kl = 1123 and 39k unknowns;
    the solve vector no longer fits in shared memory beside one factor stage, so the solves
    keep it in global scratch and read the slabs from L2; one step against the oracle."""
    w = W.config_uniform(4, 32, nsub=(2, 2), nsteps=1)
    s = native.Solver(w, precision="fp32", host_only=True)
    info = s.debug_system(0)
    assert info["kl"] == 1123 and len(info["rowptr"]) - 1 > 38000
    s.close()
    f, o, stats = run_pair(native, w, "fp32", 1, "band")
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL["fp32"], (k, rel(f[k], o.fine[k]))
    assert stats["last_ir_relres_max"] <= 1e-12


def test_band_too_wide_for_fp64_is_refused(native):
    """An FP64 panel of 32 + 851 rows does not fit one CTA's shared memory: creation fails
    with TPNS_EINVAL and a message, before any device allocation."""
    w = W.config_uniform(4, 24, nsub=(2, 2), nsteps=1)
    with pytest.raises(native.TpnsError) as e:
        native.Solver(w, precision="fp64", factor="band")
    assert e.value.status == native.TPNS_EINVAL and "shared memory" in str(e.value)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multifrontal_on_systems_too_wide_for_the_band_lu(native, prec):
    """h = 1/128 with 2 x 2 subdomains (39k-unknown Oseen systems, band kl = 1123): the
    multifrontal factorisation has no band-width limit, in FP64 as well; one step against the
    oracle."""
    w = W.config_uniform(4, 32, nsub=(2, 2), nsteps=1)
    f, o, stats = run_pair(native, w, prec, 1)
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))
    assert stats["last_ir_relres_max"] <= 1e-12


def test_multifrontal_bf16_is_refused(native):
    with pytest.raises(native.TpnsError) as e:
        native.Solver(W.config_small(nsteps=1), precision="bf16")
    assert e.value.status == native.TPNS_EINVAL


def test_multifrontal_leaf_sizes_and_launch_caps_agree(native):
    """Different dissection depths change the fronts (and so the rounding), not the result:
    every variant meets the FP32 tolerance against the oracle; a cap of 7 CTAs on the
    dataflow launches (fronts then wait for children taken by the few running CTAs) gives
    the same fields bit for bit as the default launch."""
    w = W.config_small(nsteps=3)
    o = TwoGridOracle(w)
    o.run(3)
    ref = None
    for leaf, ctas in ((0, 0), (0, 7), (24, 0), (400, 0)):
        s = native.Solver(w, precision="fp32", mf_leaf=leaf, mf_ctas=ctas)
        s.step(3)
        f = s.fields()
        s.close()
        for k in f:
            assert rel(f[k], o.fine[k]) <= TOL["fp32"], (leaf, ctas, k)
        if leaf == 0:
            if ref is None:
                ref = f
            else:
                for k in f:
                    assert np.array_equal(f[k], ref[k]), k


def test_assembled_systems_match_oracle(native):
    """FP64 CSR values and right-hand sides of the local systems after one step equal
    the oracle's assembled matrices (keyed by global node and component)."""
    w = W.config_small(nsteps=1)
    o = TwoGridOracle(w)
    d = o.step_inputs()
    s = native.Solver(w, precision="fp64")
    s.step(1)
    for j in range(len(o.sub_c) + len(o.sub_p)):
        info = s.debug_system(j)
        if j < len(o.sub_c):
            sub, O = o.sub_c[j]
            Aff, b, free, _ = o.local_fluid_system(j, d["t"], d["uH1h"], d["uH0h"], d["pH1h"], d["pFn_c"])
            nn = len(sub.gnode)
            key = [(int(sub.gnode[q // 2]), q % 2) if q < 2 * nn else (int(sub.gvert[q - 2 * nn]), 2) for q in free]
            fields = [0]
        else:
            sub, O = o.sub_p[j - len(o.sub_c)]
            fields = [0, 1, 2]
        for fld in fields:
            if j >= len(o.sub_c):
                Aff, b, free, _ = o.local_porous_system(j - len(o.sub_c), fld, d["t"], d["pdH1h"], d["pdH0h"], d["ucn_p"])
                key = [(int(sub.gnode[q]), 0) for q in free]
            pos = {k: i for i, k in enumerate(key)}
            perm = np.array([pos[(int(g), int(c))] for g, c in zip(info["node"], info["comp"])])
            vals, rhs = s.debug_values(j, fld)
            A = Aff.tocsr()
            rows = np.repeat(np.arange(len(perm)), np.diff(info["rowptr"]))
            ref_vals = np.asarray(A[perm[rows], perm[info["colidx"]]]).ravel()
            scale = np.abs(ref_vals).max()
            assert np.abs(vals - ref_vals).max() <= 1e-13 * scale, (j, fld)
            assert np.abs(rhs - b[perm]).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), (j, fld)
            # every CSR entry of the oracle is present in the library's pattern
            assert abs(A.sum() - vals.sum()) <= 1e-12 * np.abs(A).sum()
    s.close()


@pytest.mark.parametrize("factor", ["mf", "band"])
def test_deterministic_and_precomputed_coarse_path_bitwise(native, factor):
    """Two runs give bit-identical fields (no atomics in any sum), and running the local hot
    path on precomputed coarse states gives bit-identical fields to full steps."""
    w = W.config_small(nsteps=4)
    a = native.Solver(w, precision="fp32", **FACTOR[factor])
    a.step(4)
    fa = a.fields()
    a.close()
    b = native.Solver(w, precision="fp32", **FACTOR[factor])
    b.step(4)
    fb = b.fields()
    b.close()
    c = native.Solver(w, precision="fp32", **FACTOR[factor])
    c.coarse_precompute(4)
    c.local_step(4)
    fc = c.fields()
    c.close()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
        assert np.array_equal(fa[k], fc[k]), k


def test_graph_replay_equals_eager_launches_bitwise(native):
    """Steps replayed from the captured CUDA graph and steps launched kernel by kernel (per-
    phase timing on) give bit-identical fields."""
    w = W.config_small(nsteps=3)
    a = native.Solver(w, precision="fp32")
    a.step(3)
    fa = a.fields()
    a.close()
    b = native.Solver(w, precision="fp32")
    b.set_timing(True)
    b.step(3)
    fb = b.fields()
    assert b.timings()["band_lu"][1] == 3
    b.close()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_refinement_statistics(native):
    w = W.config_graded(nsteps=2)
    s = native.Solver(w, precision="fp32")
    s.step(2)
    st = s.stats()
    assert 1 <= st["last_ir_iters_max"] <= 12
    assert st["last_ir_relres_max"] <= 1e-12
    assert st["last_newton_iters"] >= 2
    s.set_timing(True)
    s.step(1)
    t = s.timings()
    assert t["band_lu"][1] == 1 and t["band_lu"][0] > 0
    s.close()


def _local_system_on_device(native, w, j, field=0):
    import torch
    s = native.Solver(w, precision="fp64")
    s.step(1)
    info = s.debug_system(j)
    vals, rhs = s.debug_values(j, field)
    s.close()
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    return info, vals, rhs, (dev(info["rowptr"], torch.int32), dev(info["colidx"], torch.int32),
                             dev(vals, torch.float64), dev(rhs, torch.float64))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("j", [0, 5], ids=["oseen", "darcy"])
def test_standalone_band_solve_matches_sparse_lu(native, prec, j):
    """tpns_band_solve on a local system of the graded workload equals SciPy's sparse LU
    of the same CSR matrix."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    import torch
    w = W.config_graded(nsteps=1) if j == 0 else W.config_small(nsteps=1)
    j_sys = 0 if j == 0 else 5                 # system 5 of the small layout is a Darcy system
    info, vals, rhs, (rp, ci, va, b) = _local_system_on_device(native, w, j_sys)
    n = len(info["node"])
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rel = native.band_solve(n, info["kl"], max(info["ku"], 1), rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                            b.data_ptr(), x.data_ptr(), precision=prec)
    assert rel <= 1e-12
    A = sps.csr_matrix((vals, info["colidx"], info["rowptr"]), shape=(n, n))
    ref = spla.splu(A.tocsc()).solve(rhs)
    got = x.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_algorithm1_on_the_same_kernels(native, prec):
    """Algorithm 1 (the partitioned time stepping on the fine grid itself) is Step 1 with the
    coarse mesh set to the fine mesh; it matches the oracle's scheme on that mesh, where the
    local corrections vanish (H = h)."""
    w = W.config_small(nsteps=3)
    o = TwoGridOracle(W.as_algorithm1(w))
    o.run(3)
    s = native.Solver(w, precision=prec, algorithm=1)
    s.step(3)
    f = s.fields()
    s.close()
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))


@pytest.mark.parametrize("prec,factor", [("fp32", "mf"), ("bf16", "band")])
def test_gmres_refinement_after_forced_stagnation(native, prec, factor):
    """One classic refinement pass per step cannot reach the tolerance; the GMRES-based
    refinement (preconditioned by the same factors, FP64 Krylov vectors) finishes every local
    system to 1e-13 within three restart cycles, and the fields meet the mixed-precision
    tolerance against the oracle."""
    w = W.config_small(nsteps=3)
    o = TwoGridOracle(w)
    o.run(3)
    s = native.Solver(w, precision=prec, gmres=True, ir_classic_max=1, **FACTOR[factor])
    s.step(3)
    f = s.fields()
    st = s.stats()
    s.close()
    assert st["gmres_steps"] >= 1 and 1 <= st["last_gmres_outer"] <= 3
    assert st["last_ir_relres_max"] <= 1e-13
    for k in f:
        assert rel(f[k], o.fine[k]) <= TOL[prec], (k, rel(f[k], o.fine[k]))


def test_gmres_refinement_idle_when_classic_converges(native):
    """With enough classic passes no GMRES cycle runs and the fields equal those of a context
    without the fallback bit for bit."""
    w = W.config_small(nsteps=2)
    a = native.Solver(w, precision="fp32", gmres=True)
    a.step(2)
    fa, st = a.fields(), a.stats()
    a.close()
    b = native.Solver(w, precision="fp32")
    b.step(2)
    fb = b.fields()
    b.close()
    assert st["gmres_steps"] == 0
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
