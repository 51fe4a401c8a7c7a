"""The multifrontal analysis of the local Oseen systems (host code, no GPU).

The library dissects each subdomain's node grid, builds the elimination tree, the update
set of every front and the maps that assemble a front from CSR values and from its
children's Schur complements.  These tests replay the numeric factorisation that the
device kernels perform -- using only the exported structure -- in NumPy, and check that it
solves the system exactly (against SciPy's sparse LU on the same matrix), together with
the structural properties every front tree must have."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W


@pytest.fixture(scope="module")
def native():
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as nat
    return nat


def _saddle_values(info, seed):
    """Random values on the pattern: velocity rows diagonally dominant, coupling to pressures
    of unit size (the pattern has no pressure-pressure block)."""
    rng = np.random.default_rng(seed)
    rp, ci, comp = info["rowptr"], info["colidx"], info["comp"]
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    v = rng.uniform(-1.0, 1.0, len(ci))
    diag = rows == ci
    v[diag & (comp[rows] < 2)] += 40.0
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def _replay(A, fr):
    """Assemble and partially factor every front in postorder exactly as the kernels do
    (unpivoted, own pivots first), then solve by the forward / backward front sweeps."""
    fronts = fr["fronts"]
    vals = A.data
    F = []
    for t, f in enumerate(fronts):
        m, p = f["m"], f["p"]
        M = np.zeros((m, m))
        for j in range(m):
            b, e = f["col_ptr"][j], f["col_ptr"][j + 1]
            M[f["orig_i"][b:e], j] = vals[f["orig_k"][b:e]]
        for c, ch in enumerate(f["children"]):
            C = fronts[ch]
            S = F[ch][C["p"]:, C["p"]:]
            for j in range(m):
                jc = f["col_child"][j, c]
                if jc >= 0:
                    M[C["relmap"], j] += S[:, jc]
        for k in range(p):
            M[k + 1:, k] /= M[k, k]
            M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
        F.append(M)
    return F


def _solve(F, fr, b):
    fronts = fr["fronts"]
    y = np.zeros_like(b)
    upd = [None] * len(fronts)
    for t, f in enumerate(fronts):
        m, p, rows = f["m"], f["p"], f["rows"]
        w = np.zeros(m)
        w[:p] = b[rows[:p]]
        for ch in f["children"]:
            w[fronts[ch]["relmap"]] += upd[ch]
        for k in range(p):
            w[k + 1:] -= F[t][k + 1:, k] * w[k]
        y[rows[:p]] = w[:p]
        upd[t] = w[p:]
    x = np.zeros_like(b)
    for t in reversed(range(len(fronts))):
        f = fronts[t]
        m, p, rows = f["m"], f["p"], f["rows"]
        w = np.concatenate([y[rows[:p]], x[rows[p:]]])
        for k in reversed(range(p)):
            w[k] = (w[k] - F[t][k, k + 1:] @ w[k + 1:]) / F[t][k, k]
        x[rows[:p]] = w[:p]
    return x


def _check_structure(fr, n):
    fronts = fr["fronts"]
    order = fr["order"]
    assert sorted(order.tolist()) == list(range(n))
    own = np.concatenate([f["rows"][:f["p"]] for f in fronts])
    assert np.array_equal(own, order)                      # postorder = elimination order
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    for t, f in enumerate(fronts):
        m, p, rows = f["m"], f["p"], f["rows"]
        assert np.all(np.diff(pos[rows[:p]]) > 0)
        if m > p:
            assert np.all(np.diff(pos[rows[p:]]) > 0) and pos[rows[p]] > pos[rows[p - 1]]
            assert f["parent"] > t
            parent = fronts[f["parent"]]
            assert np.array_equal(parent["rows"][f["relmap"]], rows[p:])
        for ch in f["children"]:
            assert fronts[ch]["parent"] == t and ch < t
            assert f["level"] > fronts[ch]["level"]


@pytest.mark.parametrize("cfg,systems", [("small", [0, 1, 2, 3]), ("graded", [0, 5])])
def test_multifrontal_structure_reproduces_sparse_solve(native, cfg, systems):
    w = W.config_small(nsteps=1) if cfg == "small" else W.config_graded(nsteps=1)
    s = native.Solver(w, host_only=True, mf_leaf=48)
    for j in systems:
        info = s.debug_system(j)
        n = len(info["node"])
        fr = s.debug_fronts(j)
        _check_structure(fr, n)
        # pressures follow the velocities inside every front
        for f in fr["fronts"]:
            c = info["comp"][f["rows"][:f["p"]]]
            assert np.all(np.diff((c == 2).astype(int)) >= 0)
        A = _saddle_values(info, seed=j)
        F = _replay(A, fr)
        b = np.random.default_rng(100 + j).standard_normal(n)
        x = _solve(F, fr, b)
        x_ref = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    s.close()


def test_planted_extend_add_mistake_is_caught(native):
    """Dropping one child's contribution (a plausible assembly bug) breaks the solve."""
    w = W.config_small(nsteps=1)
    s = native.Solver(w, host_only=True, mf_leaf=48)
    info = s.debug_system(0)
    fr = s.debug_fronts(0)
    victim = next(t for t, f in enumerate(fr["fronts"]) if len(f["children"]) == 2)
    fr["fronts"][victim]["col_child"][:, 1] = -1
    A = _saddle_values(info, seed=0)
    F = _replay(A, fr)
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    x = _solve(F, fr, b)
    x_ref = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - x_ref) > 1e-3 * np.linalg.norm(x_ref)
    s.close()


def test_band_layout_has_no_fronts(native):
    s = native.Solver(W.config_small(nsteps=1), host_only=True, factor="band")
    with pytest.raises(native.TpnsError):
        s.debug_fronts(0)
    s.close()


def test_front_table_matches_the_full_export(native):
    """The light per-front table (order, pivots, level, parent, children) equals the full
    structure export, system by system, and ends after the last Oseen system."""
    s = native.Solver(W.config_small(nsteps=1), host_only=True)
    j = 0
    while True:
        tab = s.front_table(j)
        if tab is None:
            break
        fr = s.debug_fronts(j)["fronts"]
        assert tab.shape == (len(fr), 7)
        for row, f in zip(tab.tolist(), fr):
            m, p, level, parent, nch, c0, c1 = row
            assert (m, p, level, parent) == (f["m"], f["p"], f["level"], f["parent"])
            assert [c0, c1][:nch] == f["children"]
        j += 1
    assert j == 4   # 2 x 2 conduit subdomains
    s.close()
