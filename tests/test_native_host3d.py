"""Host-side layout of the 3D configurations (no GPU): the library's Kuhn meshes, unknown
sets and CSR patterns of every local system are identical, bit for bit, to those of the
independent 3D oracle, and the multifrontal structure of 3D systems reproduces a sparse
direct solve when replayed in NumPy."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle.mesh3d import Mesh3D, region_breaks3d
from oracle.scheme3d import TwoGridOracle3D
from test_mf_host import _check_structure, _replay, _solve

CASES = [W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1),
         W.config_3d_small(n_coarse=2, r=3, nsub=(1, 2, 2), overlap=2)]


@pytest.fixture(scope="module")
def native():
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as nat
    return nat


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_meshes_bit_exact_3d(native, w):
    s = native.Solver(w, host_only=True)
    b = region_breaks3d(w)
    mc = Mesh3D(b["xs_h"], b["xs_h"], b["c"]["zs_h"])
    mp = Mesh3D(b["xs_h"], b["xs_h"], b["p"]["zs_h"])
    assert np.array_equal(s.debug_mesh(0).reshape(-1, 3), mc.node)
    assert np.array_equal(s.debug_mesh(1).reshape(-1, 3), mp.node)
    assert np.array_equal(s.debug_mesh(2).reshape(-1, 10), mc.tet10)
    assert np.array_equal(s.debug_mesh(3).reshape(-1, 10), mp.tet10)
    s.close()


def _oracle_free_sets_3d(o):
    out = []
    for s, O in o.sub_c:
        nn = len(s.gnode)
        fixed_nodes = np.nonzero(s.kind > 0)[0]
        fixed_p = 3 * nn + np.nonzero(s.art[s.vloc])[0]
        fixed = set(np.concatenate([3 * fixed_nodes, 3 * fixed_nodes + 1, 3 * fixed_nodes + 2, fixed_p]).tolist())
        key = {}
        for d in range(O.ntot):
            if d in fixed:
                continue
            key[d] = (int(s.gnode[d // 3]), d % 3) if d < 3 * nn else (int(s.gvert[d - 3 * nn]), 3)
        pairs = set()
        for e in range(len(O.vdof)):
            vel = O.vdof[e].ravel().tolist()
            pre = O.pdof[e].tolist()
            ps = set(pre)
            for r in vel + pre:
                for c in vel + pre:
                    if r in ps and c in ps:
                        continue
                    pairs.add((r, c))
        out.append((key, pairs))
    for s, O in o.sub_p:
        free = np.nonzero(s.kind == 0)[0]
        key = {int(d): (int(s.gnode[d]), 0) for d in free}
        pairs = set()
        for e in range(len(O.R.tet10)):
            nodes = O.R.tet10[e].tolist()
            pairs.update((r, c) for r in nodes for c in nodes)
        out.append((key, pairs))
    return out


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_local_unknowns_and_patterns_bit_exact_3d(native, w):
    s = native.Solver(w, host_only=True)
    o = TwoGridOracle3D(w)
    for j, (key, pairs) in enumerate(_oracle_free_sets_3d(o)):
        info = s.debug_system(j)
        mine = list(zip(info["node"].tolist(), info["comp"].tolist()))
        assert len(mine) == len(set(mine))
        assert set(mine) == set(key.values()), j
        pos = {k: i for i, k in enumerate(mine)}
        rows = np.repeat(np.arange(len(mine)), np.diff(info["rowptr"]))
        got = set(zip(rows.tolist(), info["colidx"].tolist()))
        exp = {(pos[key[r]], pos[key[c]]) for r, c in pairs if r in key and c in key}
        assert got == exp, j
    s.close()


def _saddle_values_3d(info, seed):
    """Random values on the pattern, velocity rows (components 0-2) diagonally dominant."""
    rng = np.random.default_rng(seed)
    rp, ci, comp = info["rowptr"], info["colidx"], info["comp"]
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    v = rng.uniform(-1.0, 1.0, len(ci))
    v[(rows == ci) & (comp[rows] < 3)] += 120.0
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def test_multifrontal_structure_3d_reproduces_sparse_solve(native):
    w = CASES[0]
    s = native.Solver(w, host_only=True, mf_leaf=48)
    for j in (0, 1, 3):
        info = s.debug_system(j)
        n = len(info["node"])
        fr = s.debug_fronts(j)
        _check_structure(fr, n)
        for f in fr["fronts"]:
            c = info["comp"][f["rows"][:f["p"]]]
            assert np.all(np.diff((c == 3).astype(int)) >= 0)      # pressures last in a front
        A = _saddle_values_3d(info, seed=j)
        F = _replay(A, fr)
        b = np.random.default_rng(200 + j).standard_normal(n)
        x = _solve(F, fr, b)
        x_ref = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    s.close()


def test_3d_descriptor_and_option_errors(native):
    """3D descriptors and the large-front option are validated on the host: a coarse mesh that
    is not a cube, subdomains that do not split the coarse cells, a 2D manufactured solution on
    a 3D mesh, an unknown mesh dimension and a large-front threshold below 128 are refused with
    TPNS_EINVAL before anything is allocated."""
    import ctypes as C
    lib = native.load()
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1)
    ctx = C.c_void_p()
    md, pr, pd, dd = native.descriptors(w)
    md.ny_coarse = 3
    assert lib.tpns_layout_create(C.byref(md), C.byref(pd), C.byref(ctx)) == native.TPNS_EINVAL
    md, pr, pd, dd = native.descriptors(w)
    pd.nsub_z = 3
    assert lib.tpns_layout_create(C.byref(md), C.byref(pd), C.byref(ctx)) == native.TPNS_EINVAL
    md, pr, pd, dd = native.descriptors(w)
    md.dim = 5
    assert lib.tpns_layout_create(C.byref(md), C.byref(pd), C.byref(ctx)) == native.TPNS_EINVAL
    md, pr, pd, dd = native.descriptors(w)
    dd.mms_id = 1                                   # the 2D trigonometric field
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), 0.01, 0, 0, None, C.byref(ctx))
    assert st == native.TPNS_EINVAL and not ctx.value
    with pytest.raises(native.TpnsError):
        native.Solver(w, host_only=True, mf_big_m=64)
    s = native.Solver(w, host_only=True, mf_big_m=-1)   # never: accepted
    s.close()
