"""Element growth of the unpivoted LU under adverse parameters (host, no GPU).

The local Oseen factorisations pivot on the diagonal in a static order (velocities of a
front before its pressures; in the band option every vertex pressure after the velocities
of the next half-grid column).  This is safe only while the entries of the partially
eliminated matrices stay bounded.  These tests take the oracle's own local Oseen matrices
(Alg. 3 Step 3, eq. uclocalFully) with a small viscosity and a strong convecting velocity,
permute them to the library's elimination order, eliminate without pivoting in FP64 and
bound the growth factor  max_k max|A^(k)| / max|A|  (cell Peclet numbers up to about 190).  A planted order that puts a pressure
before the velocities it couples to must fail (zero pivot)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle.scheme import TwoGridOracle

GROWTH_MAX = 1.0e3


@pytest.fixture(scope="module")
def native():
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as nat
    return nat


def _growth(A):
    """Unpivoted dense LU of A in the given order; returns (growth factor, min |pivot|, LU)
    with the unit lower factor below the diagonal and the upper factor on and above it."""
    M = np.array(A, dtype=np.float64)
    a0 = np.abs(M).max()
    g = a0
    pmin = np.inf
    n = M.shape[0]
    for k in range(n - 1):
        piv = M[k, k]
        pmin = min(pmin, abs(piv))
        if piv == 0.0:
            return np.inf, 0.0, M
        l = M[k + 1:, k] / piv
        M[k + 1:, k + 1:] -= np.outer(l, M[k, k + 1:])
        M[k + 1:, k] = l
        g = max(g, np.abs(M[k + 1:, k + 1:]).max())
    pmin = min(pmin, abs(M[-1, -1]))
    return g / a0, pmin, M


def _adverse_oracle(nu, scale, dt=0.01):
    w = W.config_small(nsteps=1)
    w.params = W.Params(**{**w.params.__dict__, "nu": nu})   # small viscosity
    w.dt = dt                                                # a long step weakens the mass term
    o = TwoGridOracle(w)
    inp = o.step_inputs()
    return w, o, inp, scale


@pytest.mark.parametrize("factor", ["mf", "band"])
@pytest.mark.parametrize("nu,scale,dt", [(0.1, 10.0, 0.01), (0.01, 30.0, 0.01), (0.1, 10.0, 1.0), (0.01, 30.0, 0.1)])
def test_unpivoted_growth_bounded(native, factor, nu, scale, dt):
    w, o, inp, scale = _adverse_oracle(nu, scale, dt)
    s = native.Solver(w, host_only=True, factor=factor, mf_leaf=48)
    for j in range(len(o.sub_c)):
        sub, O = o.sub_c[j]
        Aff, b, free, xfull = o.local_fluid_system(j, inp["t"], scale * inp["uH1h"], inp["uH0h"], inp["pH1h"],
                                                   inp["pFn_c"])
        nn = len(sub.gnode)
        key = [(int(sub.gnode[d // 2]), d % 2) if d < 2 * nn else (int(sub.gvert[d - 2 * nn]), 2) for d in free]
        info = s.debug_system(j)
        mine = list(zip(info["node"].tolist(), info["comp"].tolist()))
        pos = {k: i for i, k in enumerate(mine)}
        lib_of_oracle = np.array([pos[k] for k in key])
        order = s.debug_fronts(j)["order"] if factor == "mf" else np.arange(len(mine))
        oracle_of_lib = np.empty_like(lib_of_oracle)
        oracle_of_lib[lib_of_oracle] = np.arange(len(key))
        perm = oracle_of_lib[order]                 # elimination position -> oracle free index
        Ap = Aff.toarray()[np.ix_(perm, perm)]
        g, pmin, LU = _growth(Ap)
        assert np.isfinite(g) and g <= GROWTH_MAX, (j, g)
        assert pmin > 0.0
        # the factors of the static order solve the system: same solution as SuperLU
        x_ref = spla.spsolve(Aff.tocsc(), b)
        y = sla.solve_triangular(LU, b[perm], lower=True, unit_diagonal=True)
        xp = sla.solve_triangular(LU, y, lower=False)
        x = np.empty_like(xp)
        x[perm] = xp
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    s.close()


def test_planted_pressure_first_order_breaks(native):
    """Eliminating a pressure before any velocity it couples to meets a zero pivot (the
    saddle point's zero block): the growth check sees it."""
    w, o, inp, scale = _adverse_oracle(0.1, 10.0)
    sub, O = o.sub_c[0]
    Aff, b, free, xfull = o.local_fluid_system(0, inp["t"], scale * inp["uH1h"], inp["uH0h"], inp["pH1h"],
                                               inp["pFn_c"])
    nn = len(sub.gnode)
    is_p = free >= 2 * nn
    perm = np.concatenate([np.nonzero(is_p)[0][:1], np.nonzero(~is_p)[0], np.nonzero(is_p)[0][1:]])
    g, pmin, _ = _growth(Aff.toarray()[np.ix_(perm, perm)])
    assert not np.isfinite(g) or pmin == 0.0
