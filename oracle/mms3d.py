"""Manufactured solutions of the 3D configurations and the data they induce (Sec. 2
equations; Sec. 6: data derived from the analytical solutions).

Test infrastructure (see the package docstring).

Derived symbolically with SymPy from the strong form of Sec. 2, exactly as in 2D (``mms``):
  conduit:  f_c = du/dt - div T(u, p) + (u.grad)u,  T = 2 nu D(u) - p I
  porous:   q_i = phiC_i dp_i/dt - div(k_i/mu grad p_i) + exchange terms (F-f: sigma* k_f/mu,
            f-m: sigma k_m/mu)
Gamma is z = 1 with n_c = (0,0,-1), n_p = (0,0,1) and P_tau v = (v_x, v_y, 0).  The exact
fields need not satisfy the interface conditions, so their defects are interface data:
  g_N = -n_c.T n_c - p_F/rho
  g_T = -P_tau(T n_c) - (alpha nu / sqrt(k_F)) P_tau(u + k_F/mu grad p_F)   (x, y components)
  g_F = u.n_c - k_F/mu grad p_F . n_p,  g_f = -k_f/mu grad p_f . n_p,  g_m = -k_m/mu grad p_m . n_p
entering the weak forms as -eta<g_N, v.n_c> - eta<g_T, P_tau v> and -<g_i, v_i>.

Solutions:
  2  the 3D trigonometric field (divergence free):
     u = (sin(pi x) cos(pi y) cos(pi z), cos(pi x) sin(pi y) cos(pi z), -2 cos(pi x) cos(pi y) sin(pi z)) e^-t,
     p = cos(pi x) cos(pi y) cos(pi z) e^-t,  (p_F, p_f, p_m) = (3, 2, 1) cos(pi x) cos(pi y) cos(pi z) e^-t
  4  the steady polynomial patch field  u = (x^2, y^2, -2 (x + y) z), p = x + y + z,
     p_i = c_i (x^2 + y^2 + z^2), c = (3, 2, 1) for (F, f, m)
  0  zero fields.
"""
import numpy as np
import sympy as sp

X, Y, Z, T = sp.symbols("x y z t", real=True)
V = (X, Y, Z)


def _fields(mms_id):
    pi = sp.pi
    if mms_id == 2:
        e = sp.exp(-T)
        u = (sp.sin(pi * X) * sp.cos(pi * Y) * sp.cos(pi * Z) * e,
             sp.cos(pi * X) * sp.sin(pi * Y) * sp.cos(pi * Z) * e,
             -2 * sp.cos(pi * X) * sp.cos(pi * Y) * sp.sin(pi * Z) * e)
        base = sp.cos(pi * X) * sp.cos(pi * Y) * sp.cos(pi * Z) * e
        return u, base, (3 * base, 2 * base, 1 * base)
    if mms_id == 4:
        u = (X ** 2, Y ** 2, -2 * (X + Y) * Z)
        r2 = X ** 2 + Y ** 2 + Z ** 2
        return u, X + Y + Z, (3 * r2, 2 * r2, 1 * r2)
    if mms_id == 0:
        z = sp.Integer(0)
        return (z, z, z), z, (z, z, z)
    raise ValueError(f"unknown 3D manufactured solution {mms_id}")


def _lam(expr):
    f = sp.lambdify((X, Y, Z, T), expr, "numpy")

    def g(x, y, z, t):
        x, y, z = (np.asarray(a, dtype=float) for a in (x, y, z))
        return np.broadcast_to(np.asarray(f(x, y, z, t), dtype=float), np.broadcast(x, y, z).shape).copy()
    return g


class MMS3D:
    def __init__(self, mms_id, prm):
        u, p, pd = _fields(mms_id)
        nu, mu, rho, al = (sp.Float(v, 30) for v in (prm.nu, prm.mu, prm.rho, prm.alpha))
        sig, sigs = sp.Float(prm.sigma, 30), sp.Float(prm.sigma_star, 30)
        k = [sp.Float(v, 30) for v in prm.k]
        phiC = [sp.Float(v, 30) for v in prm.phiC]
        grad = lambda s: tuple(sp.diff(s, v) for v in V)
        lap = lambda s: sum(sp.diff(s, v, 2) for v in V)
        divu = sum(sp.diff(u[a], V[a]) for a in range(3))
        f = []
        for a, ua in enumerate(u):
            conv = sum(u[c] * sp.diff(ua, V[c]) for c in range(3))
            f.append(sp.diff(ua, T) - nu * (lap(ua) + grad(divu)[a]) + grad(p)[a] + conv)
        pF, pf, pm = pd
        cFf = sigs * k[1] / mu
        cfm = sig * k[2] / mu
        q = [phiC[0] * sp.diff(pF, T) - k[0] / mu * lap(pF) + cFf * (pF - pf),
             phiC[1] * sp.diff(pf, T) - k[1] / mu * lap(pf) + cFf * (pf - pF) + cfm * (pf - pm),
             phiC[2] * sp.diff(pm, T) - k[2] / mu * lap(pm) + cfm * (pm - pf)]
        gu = [[sp.diff(u[a], V[c]) for c in range(3)] for a in range(3)]
        Tm = [[nu * (gu[a][c] + gu[c][a]) - (p if a == c else 0) for c in range(3)] for a in range(3)]
        n_c = (0, 0, -1)
        n_p = (0, 0, 1)
        Tn = [sum(Tm[a][c] * n_c[c] for c in range(3)) for a in range(3)]
        nTn = sum(n_c[a] * Tn[a] for a in range(3))
        gN = -nTn - pF / rho
        gpF = grad(pF)
        gT = [-Tn[a] - al * nu / sp.sqrt(k[0]) * (u[a] + k[0] / mu * gpF[a]) for a in range(2)]
        g1 = sum(u[a] * n_c[a] for a in range(3)) - k[0] / mu * sum(gpF[a] * n_p[a] for a in range(3))
        gf = -k[1] / mu * sum(grad(pf)[a] * n_p[a] for a in range(3))
        gm = -k[2] / mu * sum(grad(pm)[a] * n_p[a] for a in range(3))
        on_gamma = lambda e: e.subs(Z, 1)
        self._u = [_lam(e) for e in u]
        self._gu = [[_lam(sp.diff(ua, v)) for v in V] for ua in u]
        self._p = _lam(p)
        self._pd = [_lam(e) for e in pd]
        self._gpd = [[_lam(sp.diff(e, v)) for v in V] for e in pd]
        self._f = [_lam(sp.simplify(e)) for e in f]
        self._q = [_lam(sp.simplify(e)) for e in q]
        self._gN = _lam(on_gamma(gN))
        self._gT = [_lam(on_gamma(e)) for e in gT]
        self._gd = [_lam(on_gamma(g1)), _lam(on_gamma(gf)), _lam(on_gamma(gm))]
        self.steady = mms_id in (0, 4)
        self.sym = {"u": u, "p": p, "pd": pd, "f": f, "q": q}

    def u(self, x, y, z, t):
        return np.stack([g(x, y, z, t) for g in self._u], axis=-1)

    def grad_u(self, x, y, z, t):
        return np.stack([np.stack([g(x, y, z, t) for g in row], axis=-1) for row in self._gu], axis=-2)

    def p(self, x, y, z, t):
        return self._p(x, y, z, t)

    def pd(self, i, x, y, z, t):
        return self._pd[i](x, y, z, t)

    def grad_pd(self, i, x, y, z, t):
        return np.stack([g(x, y, z, t) for g in self._gpd[i]], axis=-1)

    def f(self, x, y, z, t):
        return np.stack([g(x, y, z, t) for g in self._f], axis=-1)

    def q(self, i, x, y, z, t):
        return self._q[i](x, y, z, t)

    def gN(self, x, y, t):
        return self._gN(x, y, np.ones_like(x), t)

    def gT(self, x, y, t):
        return np.stack([g(x, y, np.ones_like(x), t) for g in self._gT], axis=-1)

    def gd(self, i, x, y, t):
        return self._gd[i](x, y, np.ones_like(x), t)
