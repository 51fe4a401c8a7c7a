"""Pins of the 3D CPU oracle against facts fixed by the paper and by mathematics: the
tetrahedral quadrature's exactness, the P2 basis, the Kuhn mesh, the strong form of Sec. 2
(finite differences), the interface defects in closed form, exact reproduction of a steady
P2/P1/P2 field by Algorithm 3, zero corrections for H = h, the local Jacobian against
central differences of the residual, closed-form Gamma sums, exact prolongation of
polynomials, the glue's partition of unity and the local discrete divergence.  Planted
mistakes (on the CPU, in the oracle) show that the pins bite."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fe3d
from oracle.mesh3d import Mesh3D, region_breaks3d
from oracle.mms3d import MMS3D
from oracle import scheme3d
from oracle.scheme3d import TwoGridOracle3D, Ops3D, prolongation3d, region_whole


def _mono(a, b, c):
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


def test_tet_rule_degree5_exact_and_not_degree6():
    P, Wq = fe3d.tet_rule()
    assert len(Wq) == 27 and abs(Wq.sum() - 1 / 6) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            for c in range(6 - a - b):
                v = np.sum(Wq * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c)
                assert abs(v - _mono(a, b, c)) < 1e-15, (a, b, c)
    worst = max(abs(np.sum(Wq * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** (6 - a - b)) - _mono(a, b, 6 - a - b))
                for a in range(7) for b in range(7 - a))
    assert worst > 1e-7


def test_p2_tet_basis_nodal_and_partition_of_unity():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    nodes = np.concatenate([v, [0.5 * (v[a] + v[b]) for a, b in fe3d.EDGES]])
    N, dN = fe3d.p2_basis(nodes)
    assert np.allclose(N, np.eye(10), atol=1e-15)
    pts = np.random.default_rng(0).dirichlet(np.ones(4), size=20)[:, 1:]
    N, dN = fe3d.p2_basis(pts)
    assert np.allclose(N.sum(axis=1), 1.0) and np.allclose(dN.sum(axis=1), 0.0, atol=1e-13)
    # gradients against central differences
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (fe3d.p2_basis(pts + e)[0] - fe3d.p2_basis(pts - e)[0]) / (2 * h)
        assert np.allclose(fd, dN[:, :, d], atol=1e-8)


def test_kuhn_mesh_counts_volumes_and_conformity():
    xs = np.linspace(0, 1, 4)
    m = Mesh3D(xs, xs, 1.0 + xs)
    assert m.nn == 7 ** 3 and len(m.tet) == 6 * 27
    det, *_ = fe3d.geometry(m.vert[m.tet])
    assert np.all(np.abs(det) > 0) and abs(np.abs(det).sum() / 6 - 1.0) < 1e-14
    assert np.allclose(m.node[m.tet10[:, 4]], 0.5 * (m.node[m.tet10[:, 0]] + m.node[m.tet10[:, 1]]))
    faces = {}
    for t in m.tet:
        for f in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
            key = tuple(sorted(t[list(f)]))
            faces[key] = faces.get(key, 0) + 1
    assert set(faces.values()) == {1, 2}
    nb = sum(1 for v in faces.values() if v == 1)
    assert nb == 6 * 2 * 9                       # 6 box faces x 9 squares x 2 triangles
    # the half grid maps back to the node coordinates
    h = m.hidx
    assert np.allclose(m.node[:, 0], 0.5 * (xs[h[:, 0] // 2] + xs[(h[:, 0] + 1) // 2]))


@pytest.mark.parametrize("mms_id", [2, 4])
def test_mms3d_forcing_matches_strong_form_by_finite_differences(mms_id):
    prm = W.Params(nu=0.7, rho=1.3, mu=1.1, alpha=0.9, sigma=0.8, sigma_star=1.2,
                   phiC=(0.5, 0.7, 0.9), k=(1.5, 0.6, 0.25))
    m = MMS3D(mms_id, prm)
    rng = np.random.default_rng(7)
    X = np.array([rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9), rng.uniform(1.1, 1.9)])
    t = 0.3
    h = 1e-4
    E = np.eye(3) * h

    def D(fn, d):
        return (fn(*(X + E[d]), t) - fn(*(X - E[d]), t)) / (2 * h)

    def Dt(fn):
        return (fn(*X, t + h) - fn(*X, t - h)) / (2 * h)

    def lap(fn):
        return sum(fn(*(X + E[d]), t) - 2 * fn(*X, t) + fn(*(X - E[d]), t) for d in range(3)) / h ** 2
    u = [lambda x, y, z, tt, a=a: m.u(x, y, z, tt)[..., a] for a in range(3)]
    divu = lambda x, y, z, tt: sum(((m.u(*(np.array([x, y, z]) + E[d]), tt) -
                                     m.u(*(np.array([x, y, z]) - E[d]), tt))[d]) / (2 * h) for d in range(3))
    assert abs(divu(*X, t)) < 1e-7                     # both fields are divergence free
    uu = m.u(*X, t)
    for a in range(3):
        conv = sum(uu[c] * D(u[a], c) for c in range(3))
        expect = Dt(u[a]) - prm.nu * (lap(u[a]) + D(divu, a)) + D(m.p, a) + conv
        assert abs(m.f(*X, t)[a] - expect) < 5e-5 * max(1, abs(expect))
    X[2] -= 1.0
    pd = [lambda x, y, z, tt, i=i: m.pd(i, x, y, z, tt) for i in range(3)]
    kF, kf, km = prm.k
    cFf, cfm = prm.sigma_star * kf / prm.mu, prm.sigma * km / prm.mu
    P = [m.pd(i, *X, t) for i in range(3)]
    ex = [prm.phiC[0] * Dt(pd[0]) - kF / prm.mu * lap(pd[0]) + cFf * (P[0] - P[1]),
          prm.phiC[1] * Dt(pd[1]) - kf / prm.mu * lap(pd[1]) + cFf * (P[1] - P[0]) + cfm * (P[1] - P[2]),
          prm.phiC[2] * Dt(pd[2]) - km / prm.mu * lap(pd[2]) + cfm * (P[2] - P[1])]
    for i in range(3):
        assert abs(m.q(i, *X, t) - ex[i]) < 5e-5 * max(1, abs(ex[i]))


def test_interface_defects_3d_closed_form():
    """Trigonometric field, all parameters 1, at z = 1: u_z = 0 and d_z p = 0, so the mass and
    no-flow defects vanish; the normal stress gives g_N = (2 - 4 pi) cos(pi x) cos(pi y) e^-t and
    the tangential condition g_T = (1 - 3 pi) (sin(pi x) cos(pi y), cos(pi x) sin(pi y)) e^-t."""
    m = MMS3D(2, W.Params())
    g = np.linspace(0, 1, 7)
    x, y = np.meshgrid(g, g)
    t = 0.37
    e = math.exp(-t)
    cx, cy, sx, sy = np.cos(np.pi * x), np.cos(np.pi * y), np.sin(np.pi * x), np.sin(np.pi * y)
    assert np.allclose(m.gN(x, y, t), (2 - 4 * np.pi) * cx * cy * e, atol=1e-13)
    gT = m.gT(x, y, t)
    assert np.allclose(gT[..., 0], (1 - 3 * np.pi) * sx * cy * e, atol=1e-13)
    assert np.allclose(gT[..., 1], (1 - 3 * np.pi) * cx * sy * e, atol=1e-13)
    for i in range(3):
        assert np.allclose(m.gd(i, x, y, t), 0.0, atol=1e-13)


def _patch_deviation_3d():
    w = W.config_3d_patch()
    o = TwoGridOracle3D(w)
    o.run(2)
    ex = o.exact_fine()
    return {k: float(np.abs(o.fine[k] - ex[k]).max()) for k in o.fine}


def test_patch_field_reproduced_exactly_3d():
    for k, d in _patch_deviation_3d().items():
        assert d < 1e-11, k


@pytest.mark.parametrize("mistake", ["BJS on x only", "normal traction sign", "exchange coefficient"])
def test_patch_pin_catches_planted_mistakes_3d(monkeypatch, mistake):
    if mistake == "BJS on x only":
        good = Ops3D.oseen_matrix

        def planted(self, w_nodal):
            A = good(self, w_nodal)
            R, prm = self.R, self.prm
            bjs = prm.eta * prm.nu * prm.alpha / np.sqrt(prm.k[0])
            d = 3 * R.faces + 1
            if len(R.faces):
                A = A - scheme3d.coo_assemble(d[:, :, None], d[:, None, :], R.gamma_mass() * bjs, self.ntot)
            return A.tocsr()
        monkeypatch.setattr(Ops3D, "oseen_matrix", planted)
        # the coarse Newton uses the same Jacobian, so plant it in the residual as well
        good_r = Ops3D.ns_residual

        def planted_r(self, u, un, p, t, mms, pF_gamma):
            r = good_r(self, u, un, p, t, mms, pF_gamma)
            R, prm = self.R, self.prm
            if len(R.faces):
                bjs = prm.eta * prm.nu * prm.alpha / np.sqrt(prm.k[0])
                ry = bjs * np.einsum("fab,fb->fa", R.gamma_mass(), u[R.faces, 1])
                np.add.at(r, (3 * R.faces + 1).ravel(), -ry.ravel())
            return r
        monkeypatch.setattr(Ops3D, "ns_residual", planted_r)
    elif mistake == "normal traction sign":
        good_r = Ops3D.ns_residual

        def planted_r(self, u, un, p, t, mms, pF_gamma):
            r = good_r(self, u, un, p, t, mms, pF_gamma)
            R, prm = self.R, self.prm
            if len(R.faces):
                rz = -(prm.eta / prm.rho) * R.gamma_load(R.gamma_trace_qp(pF_gamma))
                np.add.at(r, (3 * R.faces + 2).ravel(), -2.0 * rz.ravel())
            return r
        monkeypatch.setattr(Ops3D, "ns_residual", planted_r)
    else:
        good = Ops3D.darcy_coeffs

        def planted(self):
            c = good(self)
            p = self.prm
            c[1] = (c[1][0] - p.sigma_star * p.k[1] / p.mu, c[1][1])
            return c
        monkeypatch.setattr(Ops3D, "darcy_coeffs", planted)
    assert max(_patch_deviation_3d().values()) > 1e-6


def test_H_equals_h_gives_zero_correction_3d():
    w = W.config_3d_small(n_coarse=2, r=1, nsub=(2, 1, 1), overlap=1, nsteps=2)
    o = TwoGridOracle3D(w)
    o.run(2)
    assert max(np.abs(e).max() for e in o.ec) < 1e-12
    assert max(np.abs(e).max() for e in o.ep) < 1e-12
    assert max(np.abs(d).max() for d in o.dc) < 1e-11


def _jacobian_fd_deviation(transpose_grad=False, monkeypatch=None):
    """The local Oseen matrix is the Jacobian of the conduit residual: A d against central
    differences of the residual along random directions d (exact up to rounding: the
    residual is quadratic in u)."""
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(1, 1, 1), overlap=1, nsteps=1)
    w.params = W.Params(nu=0.7, eta=1.3, rho=1.1, mu=0.9, alpha=0.8, k=(1.7, 0.5, 0.2))
    o = TwoGridOracle3D(w)
    O = o.OcH
    rng = np.random.default_rng(11)
    nn = o.mcH.nn
    u = rng.standard_normal((nn, 3))
    un = rng.standard_normal((nn, 3))
    p = rng.standard_normal(o.mcH.nv)
    pF = rng.standard_normal(nn)
    A = O.oseen_matrix(u)
    dev = 0.0
    for _ in range(3):
        du = rng.standard_normal((nn, 3))
        dp = rng.standard_normal(o.mcH.nv)
        h = 1e-3
        rp = O.ns_residual(u + h * du, un, p + h * dp, 0.2, o.mms, pF)
        rm = O.ns_residual(u - h * du, un, p - h * dp, 0.2, o.mms, pF)
        fd = (rp - rm) / (2 * h)
        Ad = A @ np.concatenate([du.ravel(), dp])
        dev = max(dev, np.abs(Ad - fd).max() / np.abs(fd).max())
    return dev


def test_local_jacobian_matches_residual_central_differences():
    assert _jacobian_fd_deviation() < 1e-9


@pytest.mark.parametrize("mistake", ["drop b_N(e, w, v)", "transposed grad w", "sign of b(v, delta)"])
def test_jacobian_pin_catches_planted_operator_mistakes(monkeypatch, mistake):
    good = fe3d.oseen_blocks

    def planted(W_, G, w, Gw, dt, prm):
        if mistake == "drop b_N(e, w, v)":
            return good(W_, G, w, np.zeros_like(Gw), dt, prm)
        if mistake == "transposed grad w":
            return good(W_, G, w, np.swapaxes(Gw, 2, 3), dt, prm)
        Kvv, Kvp, Kpv = good(W_, G, w, Gw, dt, prm)
        return Kvv, -Kvp, Kpv
    monkeypatch.setattr(fe3d, "oseen_blocks", planted)
    assert _jacobian_fd_deviation() > 1e-4


def test_gamma_loads_closed_forms_3d():
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(1, 1, 1))
    o = TwoGridOracle3D(w)
    R = region_whole(o.mph, "p")
    O = Ops3D(R, o.prm, o.dt)
    x, y = o.mph.node[:, 0], o.mph.node[:, 1]
    g = 1 + x + y ** 2                                    # a P2 trace on Gamma
    v = O.gamma_vec(R.gamma_load(R.gamma_trace_qp(g)))
    assert abs(v.sum() - (1 + 0.5 + 1 / 3)) < 1e-14
    Rc = region_whole(o.mch, "c")
    xc, yc = o.mch.node[:, 0], o.mch.node[:, 1]
    pF = xc ** 2 - 0.7 * xc + 0.3 * xc * yc + yc ** 2
    d = Rc.gamma_grad_qp(pF)
    # sum over all basis functions of <d_x pF, v> = int_0^1 pF(1, y) - pF(0, y) dy
    assert abs(Rc.gamma_load(d[..., 0]).sum() - (1 - 0.7 + 0.15)) < 1e-14
    # and of <d_y pF, v> = int_0^1 pF(x, 1) - pF(x, 0) dx
    assert abs(Rc.gamma_load(d[..., 1]).sum() - (0.15 + 1)) < 1e-14
    assert abs(Rc.gamma_load(Rc.gamma_trace_qp(pF)).sum() - (1 / 3 - 0.35 + 0.075 + 1 / 3)) < 1e-14


def test_prolongation_exact_on_polynomials_3d():
    w = W.config_3d_small(n_coarse=2, r=2)
    b = region_breaks3d(w)
    for reg in ("c", "p"):
        mH = Mesh3D(b["xs_H"], b["xs_H"], b[reg]["zs_H"])
        mh = Mesh3D(b["xs_h"], b["xs_h"], b[reg]["zs_h"])
        q = lambda X: 0.3 + 1.7 * X[:, 0] - 0.4 * X[:, 1] + 0.8 * X[:, 2] + 2.1 * X[:, 0] ** 2 - \
            1.3 * X[:, 0] * X[:, 2] + 0.9 * X[:, 1] * X[:, 2] - 0.6 * X[:, 2] ** 2
        lin = lambda X: 0.3 + 1.7 * X[:, 0] - 0.4 * X[:, 1] + 0.8 * X[:, 2]
        P2, P1 = prolongation3d(mH, mh, "p2"), prolongation3d(mH, mh, "p1")
        assert np.abs(P2 @ q(mH.node) - q(mh.node)).max() < 1e-13
        assert np.abs(P1 @ lin(mH.vert) - lin(mh.vert)).max() < 1e-13


def test_glue_is_a_partition_of_unity_3d():
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1)
    o = TwoGridOracle3D(w)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((o.mch.nn, 3))
    for (s, _), k in zip(o.sub_c, range(len(o.ec))):
        o.ec[k] = f[s.gnode]
    o.glue()
    uHh = np.stack([o.Pc2 @ o.uH[:, a] for a in range(3)], axis=1)
    assert np.abs(o.fine["ux"] - uHh[:, 0] - f[:, 0]).max() < 1e-14


def test_local_discrete_divergence_3d():
    w = W.config_3d_small(n_coarse=2, r=2, nsub=(2, 1, 1), overlap=1, nsteps=1)
    o = TwoGridOracle3D(w)
    o.run(1)
    uH1 = np.stack([o.Pc2 @ o.uH[:, a] for a in range(3)], 1)
    for (s, O), e in zip(o.sub_c, o.ec):
        ut = (uH1[s.gnode] + e)[O.R.tet10]
        _, _, Kpv = fe3d.oseen_blocks(O.R.W, O.R.G, fe3d.at_qp(ut), fe3d.grad_at_qp(O.R.G, ut), o.dt, o.prm)
        div = np.zeros(len(s.vloc))
        np.add.at(div, O.R.tet4, np.einsum("ekjb,ejb->ek", Kpv, ut))
        assert np.abs(div[~s.art[s.vloc]]).max() < 1e-12
