"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(quadrature exactness, element invariants, the strong form of Sec. 2, exact reproduction
of P2/P1 fields, H = h, a brute-force global Newton step, closed-form interface sums,
discrete mass balance, the error norms in closed form, and the convergence rates of
Theorem 5.4 / Table T1), and checks
that planted mistakes in the oracle (a dropped or transposed convection term, a flipped
coupling sign, a wrong exchange coefficient, a wrong Beavers-Joseph-Saffman edge mass,
unnormalised glue weights, a misordered P2 basis in the prolongation) break the pins meant
to catch them."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import fe, quad
from oracle.mesh import Mesh2D, region_breaks
from oracle.mms import MMS
from oracle.scheme import TwoGridOracle, Ops, region_whole

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quadrature
def _monomial_exact(a, b):
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def test_triangle_rule_degree5_exact_and_not_degree6():
    P, Wq = quad.triangle_rule7()
    assert abs(Wq.sum() - 0.5) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            v = np.sum(Wq * P[:, 0] ** a * P[:, 1] ** b)
            assert abs(v - _monomial_exact(a, b)) < 1e-15
    worst = max(abs(np.sum(Wq * P[:, 0] ** a * P[:, 1] ** (6 - a)) - _monomial_exact(a, 6 - a))
                for a in range(7))
    assert worst > 1e-6          # a degree-5 rule must miss some degree-6 monomial


def test_duffy_rule_agrees():
    P, Wq = quad.duffy_rule(4, 4)
    for a in range(6):
        for b in range(6 - a):
            assert abs(np.sum(Wq * P[:, 0] ** a * P[:, 1] ** b) - _monomial_exact(a, b)) < 1e-15


# ------------------------------------------------------------------ elements
def _rand_tris(n=5, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, 3, 2))
    det = (X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1])
    X[det < 0] = X[det < 0][:, [0, 2, 1]]
    return X


def test_p2_basis_nodal_and_partition_of_unity():
    nodes = np.array([[0, 0], [1, 0], [0, 1], [0.5, 0], [0.5, 0.5], [0, 0.5]], dtype=float)
    N, dN = fe.p2_basis(nodes)
    assert np.allclose(N, np.eye(6), atol=1e-15)
    N, dN = fe.p2_basis(fe.QP)
    assert np.allclose(N.sum(1), 1) and np.allclose(dN.sum(1), 0)


def test_element_invariants():
    X = _rand_tris()
    det, Jinv, xq, Wt = fe.geometry(X)
    G = fe.grads(Jinv, fe.DPHI)
    M = fe.mass_p2(Wt)
    K = fe.stiff_p2(Wt, G)
    assert np.allclose(M.sum((1, 2)), 0.5 * np.abs(det), rtol=1e-14)
    assert np.allclose(K.sum(2), 0, atol=1e-12)
    assert np.allclose(K, np.swapaxes(K, 1, 2), atol=1e-13)
    prm = W.Params(nu=0.7, eta=1.3)
    rng = np.random.default_rng(3)
    w = rng.normal(size=(len(X), 6, 2))
    wq, Gw = fe.at_qp(w), fe.grad_at_qp(G, w)
    Kvv, Kvp, Kpv = fe.oseen_blocks(Wt, G, None, wq, Gw, 1e30, prm)
    xn = np.concatenate([X, 0.5 * (X[:, [0, 1, 2]] + X[:, [1, 2, 0]])], axis=1)
    # rigid motion r(x) = (a - c y, b + c x): no viscous energy; the convection part
    # b_N(r, w) + b_N(w, r) is not zero, so test the viscous part alone with w = 0
    Kvv0, _, _ = fe.oseen_blocks(Wt, G, None, 0 * wq, 0 * Gw, 1e30, prm)
    r = np.stack([0.3 - 1.7 * xn[..., 1], -0.2 + 1.7 * xn[..., 0]], axis=-1)
    assert np.abs(np.einsum("eiajb,ejb->eia", Kvv0, r)).max() < 1e-12
    # b_N(w, const, v) = 0: convection of a constant field by w vanishes
    const = np.broadcast_to(np.array([0.4, -1.1]), (len(X), 6, 2))
    # (e.grad)w term is not zero for a constant e, remove it by using w = 0 gradient
    Kc, _, _ = fe.oseen_blocks(Wt, G, None, wq, 0 * Gw, 1e30, prm)
    assert np.abs(np.einsum("eiajb,ejb->eia", Kc - Kvv0, const)).max() < 1e-12
    # pressure rows: eta (q, div u) for u = (x, 2y): div u = 3 -> 3 eta |K|/3 per vertex
    u = np.stack([xn[..., 0], 2 * xn[..., 1]], axis=-1)
    got = np.einsum("ekjb,ejb->ek", Kpv, u)
    assert np.allclose(got, prm.eta * 3 * (0.5 * np.abs(det))[:, None] / 3, rtol=1e-13)
    # velocity-pressure block is minus the transpose of the pressure rows
    assert np.allclose(Kvp, -np.transpose(Kpv, (0, 2, 3, 1)), atol=1e-14)


# ------------------------------------------------------------------ manufactured data
@pytest.mark.parametrize("mms_id", [1, 3])
def test_mms_forcing_matches_strong_form_by_finite_differences(mms_id):
    prm = W.Params(nu=0.7, rho=1.3, mu=1.1, alpha=0.9, sigma=0.8, sigma_star=1.2,
                   phiC=(0.5, 0.7, 0.9), k=(1.5, 0.6, 0.25))
    m = MMS(mms_id, prm)
    rng = np.random.default_rng(5)
    x, y, t = rng.uniform(0.1, 0.9), rng.uniform(1.1, 1.9), 0.3
    h = 1e-4

    def d(fn, var, *args):
        if var == "x":
            return (fn(x + h, y, t) - fn(x - h, y, t)) / (2 * h)
        if var == "y":
            return (fn(x, y + h, t) - fn(x, y - h, t)) / (2 * h)
        return (fn(x, y, t + h) - fn(x, y, t - h)) / (2 * h)

    def lap(fn):
        return ((fn(x + h, y, t) - 2 * fn(x, y, t) + fn(x - h, y, t)) +
                (fn(x, y + h, t) - 2 * fn(x, y, t) + fn(x, y - h, t))) / h ** 2
    u = lambda a: (lambda X_, Y_, T_: m.u(X_, Y_, T_)[..., a])
    divu = lambda X_, Y_, T_: (m.u(X_ + h, Y_, T_)[..., 0] - m.u(X_ - h, Y_, T_)[..., 0]) / (2 * h) + \
        (m.u(X_, Y_ + h, T_)[..., 1] - m.u(X_, Y_ - h, T_)[..., 1]) / (2 * h)
    uu = m.u(x, y, t)
    for a, var in enumerate("xy"):
        conv = uu[0] * d(u(a), "x") + uu[1] * d(u(a), "y")
        expect = d(u(a), "t") - prm.nu * (lap(u(a)) + d(divu, var)) + d(m.p, var) + conv
        assert abs(m.f(x, y, t)[a] - expect) < 2e-5 * max(1, abs(expect))
    yp = y - 1.0
    pd = [lambda X_, Y_, T_, i=i: m.pd(i, X_, Y_, T_) for i in range(3)]
    kF, kf, km = prm.k
    cFf, cfm = prm.sigma_star * kf / prm.mu, prm.sigma * km / prm.mu
    y = yp
    P = [m.pd(i, x, y, t) for i in range(3)]
    ex = [prm.phiC[0] * d(pd[0], "t") - kF / prm.mu * lap(pd[0]) + cFf * (P[0] - P[1]),
          prm.phiC[1] * d(pd[1], "t") - kf / prm.mu * lap(pd[1]) + cFf * (P[1] - P[0]) + cfm * (P[1] - P[2]),
          prm.phiC[2] * d(pd[2], "t") - km / prm.mu * lap(pd[2]) + cfm * (P[2] - P[1])]
    for i in range(3):
        assert abs(m.q(i, x, y, t) - ex[i]) < 2e-5 * max(1, abs(ex[i]))


def test_interface_defects_closed_form():
    json.load(open(os.path.join(GOLD, "interface_closed_forms.json")))
    m = MMS(1, W.Params())
    x = np.linspace(0, 1, 9)
    t = 0.37
    e = math.exp(-t)
    assert np.allclose(m.gN(x, t), (-(2 * np.pi + 1) + 3) * np.cos(np.pi * x) * e, atol=1e-14)
    assert np.allclose(m.gT(x, t), (1 - 3 * np.pi) * np.sin(np.pi * x) * e, atol=1e-13)
    assert np.allclose(m.gd(0, x, t), 0, atol=1e-14)


# ------------------------------------------------------------------ meshes
def test_mesh_counts_and_nesting():
    w = W.config_small()
    b = region_breaks(w)
    mc = Mesh2D(b["xs_h"], b["c"]["ys_h"])
    mp = Mesh2D(b["xs_h"], b["p"]["ys_h"])
    assert 2 * mc.nn + mc.nv == 2467 and 3 * mp.nn == 3267
    assert set(b["xs_H"]).issubset(set(b["xs_h"]))
    assert set(b["c"]["ys_H"]).issubset(set(b["c"]["ys_h"]))
    # edge nodes are midpoints, edges sorted lexicographically
    assert (np.diff(mc.edges[:, 0]) >= 0).all()
    for m in (mc, mp):
        t6 = m.tri6
        assert np.allclose(m.node[t6[:, 3]], 0.5 * (m.node[t6[:, 0]] + m.node[t6[:, 1]]))
        X = m.tri_coords()
        det, *_ = fe.geometry(X)
        assert (det > 0).all()
    g = W.config_graded()
    bg = region_breaks(g)
    assert len(bg["c"]["ys_h"]) == 49 and abs(bg["c"]["ys_h"][1] - 1 - 1 / 128) < 1e-15
    assert abs(bg["p"]["ys_h"][1] - 1 / 32) < 1e-15


# ------------------------------------------------------------------ exact reproduction
def _patch_deviation(graded):
    """Largest deviation, per field, of Algorithm 3's fine fields from a steady field with P2
    velocity, P1 pressure and P2 Darcy pressures after three steps."""
    w = W.config_patch(nx_coarse=2, r=2, nsub=(2, 2), nsteps=3)
    if graded:
        w.nx_coarse, w.ny_coarse, w.fine_per_coarse_x = 4, 4, 2
        w.fine_rows_from_gamma = [4, 2, 1, 1]
    o = TwoGridOracle(w)
    o.run(3)
    ex = o.exact_fine()
    return {k: float(np.abs(o.fine[k] - ex[k]).max()) for k in o.fine}


@pytest.mark.parametrize("graded", [False, True])
def test_patch_field_reproduced_exactly(graded):
    """The steady P2/P1 field is reproduced by Algorithm 3 at every step (backward Euler and
    all lagging are exact for it)."""
    for k, d in _patch_deviation(graded).items():
        assert d < 1e-11, k


def test_H_equals_h_gives_zero_correction():
    w = W.config_uniform(4, 1, nsub=(2, 2), overlap=1, nsteps=2)
    o = TwoGridOracle(w)
    o.run(2)
    assert max(np.abs(e).max() for e in o.ec) < 1e-12
    assert max(np.abs(e).max() for e in o.ep) < 1e-12
    assert max(np.abs(d).max() for d in o.dc) < 1e-11


# ------------------------------------------------------------------ prolongation (Step 3 data)
def _prolongation_deviation(graded):
    """Nested meshes: the fine interpolant of a coarse P2 (P1) function is that function, so
    prolongating the coarse nodal values of a quadratic (linear) polynomial must give its
    values at the fine nodes (vertices) exactly."""
    from oracle.scheme import prolongation
    w = W.config_graded() if graded else W.config_uniform(4, 2, nsub=(2, 2))
    b = region_breaks(w)
    dev = 0.0
    for reg in ("c", "p"):
        mH, mh = Mesh2D(b["xs_H"], b[reg]["ys_H"]), Mesh2D(b["xs_h"], b[reg]["ys_h"])

        def q(x, y):
            return 0.3 + 1.7 * x - 0.4 * y + 2.1 * x * x - 1.3 * x * y + 0.9 * y * y

        def l(x, y):
            return 0.3 + 1.7 * x - 0.4 * y

        P2, P1 = prolongation(mH, mh, "p2"), prolongation(mH, mh, "p1")
        dev = max(dev, np.abs(P2 @ q(mH.node[:, 0], mH.node[:, 1]) - q(mh.node[:, 0], mh.node[:, 1])).max(),
                  np.abs(P1 @ l(mH.vert[:, 0], mH.vert[:, 1]) - l(mh.vert[:, 0], mh.vert[:, 1])).max())
    return dev


@pytest.mark.parametrize("graded", [False, True])
def test_prolongation_exact_on_polynomials(graded):
    assert _prolongation_deviation(graded) < 1e-13


def test_prolongation_pin_catches_planted_basis_order(monkeypatch):
    """The two last P2 basis functions (edge midpoints) swapped."""
    good = fe.p2_basis

    def planted(pts):
        N, dN = good(pts)
        return N[:, [0, 1, 2, 3, 5, 4]], dN

    monkeypatch.setattr(fe, "p2_basis", planted)
    assert _prolongation_deviation(False) > 1e-3


# ------------------------------------------------------------------ glue (Step 4)
def _glue_deviation():
    """Corrections that all restrict one fine field g (velocity, pressure and the three Darcy
    pressures) must glue to I_h u_H + g: the weights form a partition of unity over the D_j
    covering each node (4 x 2 fluid and porous subdomains, overlapping)."""
    w = W.config_uniform(4, 2, nsub=(4, 2), overlap=3, nsteps=1)
    o = TwoGridOracle(w)
    rng = np.random.default_rng(0)
    gu = rng.standard_normal((o.mch.nn, 2))
    gp = rng.standard_normal(o.mch.nv)
    gd = rng.standard_normal((3, o.mph.nn))
    o.ec = [gu[s.gnode] for (s, _) in o.sub_c]
    o.dc = [gp[s.gvert] for (s, _) in o.sub_c]
    o.ep = [gd[:, s.gnode] for (s, _) in o.sub_p]
    f = o.glue()
    dev = [np.abs(f["ux"] - o.Pc2 @ o.uH[:, 0] - gu[:, 0]).max(),
           np.abs(f["uy"] - o.Pc2 @ o.uH[:, 1] - gu[:, 1]).max(),
           np.abs(f["p"] - o.Pc1 @ o.pH - gp).max()]
    dev += [np.abs(f[k] - o.Pp2 @ o.pdH[i] - gd[i]).max() for i, k in enumerate(("pF", "pf", "pm"))]
    return max(dev)


def test_glue_is_a_partition_of_unity():
    assert _glue_deviation() < 1e-14


def test_glue_pin_catches_planted_unnormalised_weights(monkeypatch):
    """Weights of 1 on every D_j instead of 1 / (number of D_j holding the node)."""
    monkeypatch.setattr(TwoGridOracle, "_pou", staticmethod(lambda subs, nn: np.ones(nn)))
    assert _glue_deviation() > 0.1


# ------------------------------------------------------------------ brute force
def _newton_step_deviation():
    """Largest deviations (velocity, pressure, Darcy pressures) of the oracle's step from one
    Newton step of the global fine backward-Euler problem (see the test below)."""
    w = W.config_uniform(2, 2, nsub=(1, 1), overlap=1, nsteps=1, dt=0.05)
    o = TwoGridOracle(w)
    prev = dict(o.fine)
    uH0, pdH0 = o.uH.copy(), o.pdH.copy()
    o.step()
    t = o.dt
    m = o.mms
    R = region_whole(o.mch, "c")
    O = Ops(R, o.prm, o.dt)
    nn = o.mch.nn
    un = np.stack([prev["ux"], prev["uy"]], axis=1)
    pF = np.zeros(nn)
    pF[o.gam_c_h] = (o.Pp2 @ pdH0[0])[o.gam_p_h]
    # linearisation point: the fine interpolant of the new coarse solution
    x0 = np.concatenate([np.stack([o.Pc2 @ o.uH[:, a] for a in range(2)], 1).ravel(), o.Pc1 @ o.pH])
    d = o._region_dirichlet(o.mch, "c")
    ub = m.u(o.mch.node[d, 0], o.mch.node[d, 1], t)
    fixed = np.concatenate([2 * d, 2 * d + 1])
    dB = np.concatenate([ub[:, 0], ub[:, 1]]) - x0[fixed]      # boundary step to the fine data
    free = np.setdiff1d(np.arange(O.ntot), fixed)

    def F(x):
        return O.ns_residual(x[:2 * nn].reshape(nn, 2), un, x[2 * nn:], t, m, pF)
    J = np.zeros((O.ntot, O.ntot))
    hstep = 1e-3
    for k in range(O.ntot):
        xp, xm = x0.copy(), x0.copy()
        xp[k] += hstep
        xm[k] -= hstep
        J[:, k] = (F(xp) - F(xm)) / (2 * hstep)
    x = x0.copy()
    x[fixed] += dB
    x[free] += np.linalg.solve(J[np.ix_(free, free)], -F(x0)[free] - J[np.ix_(free, fixed)] @ dB)
    u_bf = x[:2 * nn].reshape(nn, 2)
    du = max(np.abs(u_bf[:, 0] - o.fine["ux"]).max(), np.abs(u_bf[:, 1] - o.fine["uy"]).max())
    dpr = np.abs(x[2 * nn:] - o.fine["p"]).max()
    # Darcy: the fine backward-Euler step with partners lagged at the fine state
    Rp = region_whole(o.mph, "p")
    Op = Ops(Rp, o.prm, o.dt)
    Mf = Op.mass_matrix().toarray()
    pn = np.stack([prev["pF"], prev["pf"], prev["pm"]])
    prm = o.prm
    kF, kf, km = prm.k
    cFf, cfm = prm.sigma_star * kf / prm.mu, prm.sigma * km / prm.mu
    partners = {0: [(cFf, 1)], 1: [(cfm, 2), (cFf, 0)], 2: [(cfm, 1)]}
    ucn = np.zeros(o.mph.nn)
    ucn[o.gam_p_h] = -(o.Pc2 @ uH0[:, 1])[o.gam_c_h]
    dp = o._region_dirichlet(o.mph, "p")
    freep = np.setdiff1d(np.arange(o.mph.nn), dp)
    dd = 0.0
    for i, key in enumerate(("pF", "pf", "pm")):
        A = Op.darcy_matrix(i).toarray()
        b = Op.darcy_load(m.q(i, Rp.xq[..., 0], Rp.xq[..., 1], t)) + prm.phiC[i] / o.dt * Mf @ pn[i]
        for c, k in partners[i]:
            b += c * Mf @ pn[k]
        if i == 0:
            b += Op.gamma_vec(Rp.gamma_load(Rp.gamma_trace_qp(ucn)))
        b -= Op.gamma_vec(Rp.gamma_load(m.gd(i, Rp.exq, t)))
        x = np.zeros(o.mph.nn)
        x[dp] = m.pd(i, o.mph.node[dp, 0], o.mph.node[dp, 1], t)
        x[freep] = np.linalg.solve(A[np.ix_(freep, freep)], b[freep] - A[np.ix_(freep, dp)] @ x[dp])
        dd = max(dd, np.abs(x - o.fine[key]).max())
    return du, dpr, dd


def test_single_subdomain_equals_global_newton_step():
    """With one subdomain per region, u_H + e is one Newton step of the global fine
    backward-Euler problem about the coarse solution (coarse Gamma data).  The Jacobian
    is formed by central differences of the residual (exact for a quadratic residual) and
    the step solved densely with numpy.linalg.solve."""
    du, dp, dd = _newton_step_deviation()
    assert du < 1e-10 and dp < 1e-9 and dd < 1e-11


# ------------------------------------------------------------------ planted mistakes
# Each test plants one plausible mistake in the oracle (on the CPU, for this test only) and
# checks that the pin meant to guard against it no longer holds.
@pytest.mark.parametrize("mistake", ["drop b_N(e, w, v)", "sign of b(v, delta)", "transposed grad w"])
def test_newton_pin_catches_planted_operator_mistakes(monkeypatch, mistake):
    good = fe.oseen_blocks

    def planted(W_, G, GP, w, Gw, dt, prm):
        if mistake == "drop b_N(e, w, v)":
            return good(W_, G, GP, w, np.zeros_like(Gw), dt, prm)
        if mistake == "transposed grad w":
            return good(W_, G, GP, w, np.swapaxes(Gw, 2, 3), dt, prm)
        Kvv, Kvp, Kpv = good(W_, G, GP, w, Gw, dt, prm)
        return Kvv, -Kvp, Kpv

    monkeypatch.setattr(fe, "oseen_blocks", planted)
    try:
        du, dp, _ = _newton_step_deviation()
    except (ArithmeticError, np.linalg.LinAlgError, RuntimeError):
        return                                   # the scheme broke down: caught as well
    assert max(du, dp) > 1e-6


@pytest.mark.parametrize("mistake", ["exchange coefficient", "Gamma edge mass"])
def test_patch_pin_catches_planted_coefficient_mistakes(monkeypatch, mistake):
    """Dropping the sigma* k_f / mu part of the fracture pressure's exchange coefficient
    (the coefficient c_f of the second Darcy equation), or doubling the Gamma edge mass that
    carries the Beavers-Joseph-Saffman term."""
    from oracle import scheme
    if mistake == "exchange coefficient":
        good = Ops.darcy_coeffs

        def planted(self):
            c = good(self)
            p = self.prm
            c[1] = (c[1][0] - p.sigma_star * p.k[1] / p.mu, c[1][1])
            return c

        monkeypatch.setattr(Ops, "darcy_coeffs", planted)
    else:
        good_m = scheme.Region.gamma_mass
        monkeypatch.setattr(scheme.Region, "gamma_mass", lambda self: 2.0 * good_m(self))
    assert max(_patch_deviation(False).values()) > 1e-6


# ------------------------------------------------------------------ closed-form interface sums
def test_gamma_loads_closed_forms():
    w = W.config_uniform(2, 4, nsub=(1, 1))
    o = TwoGridOracle(w)
    R = region_whole(o.mph, "p")
    O = Ops(R, o.prm, o.dt)
    xs = o.mph.node[:, 0]
    # sum over all P2 basis functions of <g, v> is int_Gamma g (partition of unity)
    g = 1 + xs + xs ** 2                                      # a P2 trace on Gamma
    v = O.gamma_vec(R.gamma_load(R.gamma_trace_qp(g)))
    assert abs(v.sum() - (1 + 0.5 + 1 / 3)) < 1e-14
    # BJS coupling: sum over tangential components of <d_tau p, v.tau> = p(1,1) - p(0,1)
    Rc = region_whole(o.mch, "c")
    pFg = np.zeros(o.mch.nn)
    xc = o.mch.node[:, 0]
    pFg[:] = np.cos(1.3 * xc) * 0 + xc ** 2 - 0.7 * xc
    dv = Rc.gamma_load(Rc.gamma_dtau_qp(pFg))
    assert abs(dv.sum() - ((1 - 0.7) - 0.0)) < 1e-14
    # normal traction: sum of <p_F, v.n_c> over v_y = -int p_F
    tv = Rc.gamma_load(Rc.gamma_trace_qp(pFg))
    assert abs(tv.sum() - (1 / 3 - 0.35)) < 1e-14


# ------------------------------------------------------------------ discrete mass balance
def test_local_discrete_divergence():
    w = W.config_small(nsteps=2)
    o = TwoGridOracle(w)
    o.run(1)
    uH1 = np.stack([o.Pc2 @ o.uH[:, a] for a in range(2)], 1)
    for (s, O), e in zip(o.sub_c, o.ec):
        utot = (uH1[s.gnode] + e)[O.R.tri6]
        wq = fe.at_qp(utot)
        _, _, Kpv = fe.oseen_blocks(O.R.W, O.R.G, None, wq, fe.grad_at_qp(O.R.G, utot), o.dt, o.prm)
        div = np.zeros(len(s.vloc))
        np.add.at(div, O.R.tri3, np.einsum("ekjb,ejb->ek", Kpv, utot))
        test = ~s.art[s.vloc]                   # pressure tests of Q_0^h(Omega_j)
        assert np.abs(div[test]).max() < 1e-12


# ------------------------------------------------------------------ convergence rates
@pytest.mark.slow
def test_convergence_rates_theorem_5_4():
    """Rates of Algorithm 3 with h = H^2 and the paper's overlap of 1/4 (Example 1
    layout), small dt so that the time error stays below the spatial error."""
    gold = json.load(open(os.path.join(GOLD, "paper_rates.json")))
    res = []
    for H, r in [(4, 4), (8, 8)]:
        w = W.config_uniform(H, r, nsub=(2, 2), overlap=(H * r) // 4, nsteps=2, dt=1e-4)
        o = TwoGridOracle(w)
        o.run(2)
        res.append(o.errors())
    rate = lambda k: math.log(res[0][k] / res[1][k]) / math.log(4)
    assert rate("u_H1") >= gold["min_velocity_H1_rate"]
    for k in ("pF_L2", "pf_L2", "pm_L2"):
        assert rate(k) >= gold["min_darcy_L2_rate"]


@pytest.mark.slow
def test_algorithm3_approaches_algorithm1_as_H_shrinks():
    """Algorithms 3 and 1 differ by the two-grid error c (dt + H^{r+1}) (Sec. 5 vs Sec. 3.3;
    compare Tables 1 and 2 of Sec. 6): halving H (h = H/4, dt fixed) shrinks the difference by
    more than 3 in every field, and at H = 1/8 the difference is below the larger of the two
    schemes' own errors against the exact solution (the schemes agree to their accuracy)."""
    import numpy as np
    diffs = []
    for nx in (4, 8):
        w = W.config_uniform(nx, 4, nsub=(2, 2), overlap=2, dt=0.01, nsteps=5)
        o3 = TwoGridOracle(w)
        o3.run(5)
        o1 = TwoGridOracle(W.as_algorithm1(w))
        o1.run(5)
        ex = o3.exact_fine()
        d = {k: np.linalg.norm(o3.fine[k] - o1.fine[k]) / np.linalg.norm(ex[k]) for k in ex}
        e1 = {k: np.linalg.norm(o1.fine[k] - ex[k]) / np.linalg.norm(ex[k]) for k in ex}
        e3 = {k: np.linalg.norm(o3.fine[k] - ex[k]) / np.linalg.norm(ex[k]) for k in ex}
        diffs.append(d)
    for k in diffs[0]:
        assert diffs[0][k] > 3.0 * diffs[1][k], k
        assert diffs[1][k] < max(e1[k], e3[k]), k


# ------------------------------------------------------------------ error norms
def test_error_norms_match_closed_forms():
    """The error norms the rate test reads (velocity H1 and L2, pressure L2, Darcy L2 and
    H1): zero for the exact polynomial patch field, and for fields shifted by a constant or
    a linear function the closed forms over the unit-area regions (fluid [0,1]x[1,2], porous
    [0,1]^2): a constant c in a pressure gives an L2 error |c|; a*x added to u_x gives an H1
    seminorm |a| and an L2 norm |a|/sqrt(3); b*y added to p_F gives an H1 seminorm |b| and an
    L2 norm |b|/sqrt(3)."""
    o = TwoGridOracle(W.config_patch(nx_coarse=2, r=3, nsub=(1, 1), nsteps=1))
    o.fine = o.exact_fine()
    base = o.errors()
    assert set(base) == {"u_H1", "u_L2", "p_L2", "pF_L2", "pF_H1", "pf_L2", "pf_H1", "pm_L2", "pm_H1"}
    assert max(base.values()) < 1e-12, base
    a, c, b, d = 0.7, -0.3, 1.9, 0.45
    f = o.exact_fine()
    f["ux"] = f["ux"] + a * o.mch.node[:, 0]
    f["p"] = f["p"] + c
    f["pF"] = f["pF"] + b * o.mph.node[:, 1]
    f["pm"] = f["pm"] + d
    o.fine = f
    e = o.errors()
    expect = {"u_H1": abs(a), "u_L2": abs(a) / math.sqrt(3.0), "p_L2": abs(c), "pF_L2": abs(b) / math.sqrt(3.0),
              "pF_H1": abs(b), "pf_L2": 0.0, "pf_H1": 0.0, "pm_L2": abs(d), "pm_H1": 0.0}
    for k, v in expect.items():
        assert abs(e[k] - v) < 1e-12, (k, e[k], v)
