"""CPU tests of the native library: it builds for sm_103a and exports every symbol its
header declares; meshes, unknown sets and CSR patterns built by the library's host code
are identical, bit for bit, to those of the independent oracle; argument errors are
reported as status codes.  No kernel runs here (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.mesh import Mesh2D, region_breaks
from oracle.scheme import TwoGridOracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as N
    N.load()
    return N


def test_library_exports_every_declared_symbol(native):
    hdr = open(os.path.join(ROOT, "include", "tpns.h")).read()
    declared = set(re.findall(r"\b(tpns_[a-z_]+)\s*\(", hdr))
    assert "tpns_create" in declared and "tpns_step" in declared
    lib = native.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
        C.cast(getattr(lib, name), C.c_void_p)      # resolvable
    assert set(native.EXPORTS) >= declared


WORKLOADS = [W.config_small(), W.config_graded(), W.config_patch(), W.config_uniform(4, 2, nsub=(1, 1)),
             W.config_uniform(8, 2, nsub=(4, 2), overlap=3)]


@pytest.mark.parametrize("w", WORKLOADS, ids=lambda w: w.name)
def test_meshes_bit_exact(native, w):
    s = native.Solver(w, host_only=True)
    b = region_breaks(w)
    mc = Mesh2D(b["xs_h"], b["c"]["ys_h"])
    mp = Mesh2D(b["xs_h"], b["p"]["ys_h"])
    assert np.array_equal(s.debug_mesh(0).reshape(-1, 2), mc.node)
    assert np.array_equal(s.debug_mesh(1).reshape(-1, 2), mp.node)
    assert np.array_equal(s.debug_mesh(2).reshape(-1, 6), mc.tri6)
    assert np.array_equal(s.debug_mesh(3).reshape(-1, 6), mp.tri6)
    s.close()


def _oracle_free_sets(o):
    """Unknowns and structural sparsity of every local system of the oracle, keyed by
    (global node, component); Oseen systems first, then one pattern per porous subdomain.
    The structure is the union over elements of their (test, trial) unknown pairs, without
    the pressure-pressure block."""
    out = []
    for s, O in o.sub_c:
        nn = len(s.gnode)
        fixed_nodes = np.nonzero(s.kind > 0)[0]
        fixed_p = 2 * nn + np.nonzero(s.art[s.vloc])[0]
        fixed = set(np.concatenate([2 * fixed_nodes, 2 * fixed_nodes + 1, fixed_p]).tolist())
        key = {}
        for d in range(O.ntot):
            if d in fixed:
                continue
            key[d] = (int(s.gnode[d // 2]), d % 2) if d < 2 * nn else (int(s.gvert[d - 2 * nn]), 2)
        pairs = set()
        for e in range(len(O.vdof)):
            vel = O.vdof[e].ravel().tolist()
            pre = O.pdof[e].tolist()
            for r in vel + pre:
                for c in vel + pre:
                    if r in pre and c in pre:
                        continue
                    pairs.add((r, c))
        out.append((key, pairs))
    for s, O in o.sub_p:
        free = np.nonzero(s.kind == 0)[0]
        key = {int(d): (int(s.gnode[d]), 0) for d in free}
        pairs = set()
        for e in range(len(O.R.tri6)):
            nodes = O.R.tri6[e].tolist()
            pairs.update((r, c) for r in nodes for c in nodes)
        out.append((key, pairs))
    return out


@pytest.mark.parametrize("w", [W.config_small(), W.config_graded(), W.config_uniform(8, 2, nsub=(4, 2), overlap=3)],
                         ids=lambda w: w.name)
def test_local_unknowns_and_patterns_bit_exact(native, w):
    s = native.Solver(w, host_only=True)
    o = TwoGridOracle(w)
    ref = _oracle_free_sets(o)
    for j, (key, pairs) in enumerate(ref):
        info = s.debug_system(j)
        mine = list(zip(info["node"].tolist(), info["comp"].tolist()))
        assert len(mine) == len(set(mine))
        assert set(mine) == set(key.values()), j
        pos = {k: i for i, k in enumerate(mine)}
        rows = np.repeat(np.arange(len(mine)), np.diff(info["rowptr"]))
        got = set(zip(rows.tolist(), info["colidx"].tolist()))
        exp = {(pos[key[r]], pos[key[c]]) for r, c in pairs if r in key and c in key}
        assert got == exp, j
        # band widths are those of the pattern
        assert info["kl"] == max(r - c for r, c in got) and info["ku"] == max(c - r for r, c in got)
    s.close()


def test_band_order_puts_pressures_after_next_column(native):
    """The unpivoted band LU relies on every vertex pressure following the velocities of
    the next half-grid column (so that leading blocks stay invertible)."""
    w = W.config_small()
    s = native.Solver(w, host_only=True)
    b = region_breaks(w)
    mc = Mesh2D(b["xs_h"], b["c"]["ys_h"])
    I_of = np.zeros(mc.nn, dtype=int)
    J_of = np.zeros(mc.nn, dtype=int)
    for J in range(mc.half.shape[0]):
        for I in range(mc.half.shape[1]):
            I_of[mc.half[J, I]] = I
            J_of[mc.half[J, I]] = J
    o = TwoGridOracle(w)
    for j, (sub, _) in enumerate(o.sub_c):
        info = s.debug_system(j)
        along_x = (sub.i1 - sub.i0) >= (sub.j1 - sub.j0)
        col = I_of[info["node"]] if along_x else J_of[info["node"]]
        vel = info["comp"] < 2
        pos = np.arange(len(col))
        for k in np.nonzero(~vel)[0]:
            C_ = col[k]
            before = pos[vel & (col <= C_ + 1)]
            after = pos[vel & (col >= C_ + 2)]
            assert before.size == 0 or before.max() < k
            assert after.size == 0 or after.min() > k
    s.close()


def test_invalid_arguments_are_status_codes(native):
    w = W.config_small()
    md, pr, pd, dd = native.descriptors(w)
    lib = native.load()
    ctx = C.c_void_p()
    pr.nu = -1.0
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), 0.01, 0, 0, None, C.byref(ctx))
    assert st == native.TPNS_EINVAL and not ctx.value
    assert b"parameters" in lib.tpns_last_error(None)
    md, pr, pd, dd = native.descriptors(w)
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), -0.01, 0, 0, None, C.byref(ctx))
    assert st == native.TPNS_EINVAL
    pd.nsub_x = 3                                  # does not split 4 coarse columns
    st = lib.tpns_layout_create(C.byref(md), C.byref(pd), C.byref(ctx))
    assert st == native.TPNS_EINVAL
    md, pr, pd, dd = native.descriptors(w)
    dd.mms_id = 7
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), 0.01, 0, 0, None, C.byref(ctx))
    assert st == native.TPNS_EINVAL
    # calls that need device state are refused on a host-only context
    s = native.Solver(w, host_only=True)
    assert lib.tpns_step(s.ctx, 1) == native.TPNS_EINVAL
    assert lib.tpns_set_timing(s.ctx, 1) == native.TPNS_EINVAL
    # a batched step with a host-only context (or a NULL one, or a negative count) is refused
    # before anything is enqueued
    arr = (C.c_void_p * 2)(s.ctx, None)
    assert lib.tpns_batch_step(arr, 1) == native.TPNS_EINVAL
    assert lib.tpns_batch_step(arr, 2) == native.TPNS_EINVAL
    assert lib.tpns_batch_step(arr, -1) == native.TPNS_EINVAL
    assert lib.tpns_batch_step(None, 1) == native.TPNS_EINVAL
    s.close()
    # the precisions outside the enum are refused
    md, pr, pd, dd = native.descriptors(w)
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), 0.01, 9, 0, None, C.byref(ctx))
    assert st == native.TPNS_EINVAL


def test_budget_refusal_before_any_allocation(native):
    """An HBM budget smaller than the footprint is refused with TPNS_EBUDGET before any
    device allocation (so it is testable without a GPU)."""
    w = W.config_graded()
    md, pr, pd, dd = native.descriptors(w)
    lib = native.load()
    ctx = C.c_void_p()
    st = lib.tpns_create(C.byref(md), C.byref(pr), C.byref(pd), C.byref(dd), 0.005, 1, 1 << 20, None, C.byref(ctx))
    assert st == native.TPNS_EBUDGET, native.STATUS_NAMES[st]
    assert b"budget" in lib.tpns_last_error(None)
