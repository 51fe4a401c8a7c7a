"""Manufactured solutions and the data they induce (Sec. 2 equations, Sec. 6 usage:
"initial conditions, boundary conditions and forcing terms are derived from the
analytical solutions").

Derived symbolically with SymPy from the strong form of Sec. 2:
  conduit:  f_c = du/dt - div T(u, p) + (u.grad)u,  T = 2 nu D(u) - p I
  porous:   q_F = phiC_F dp_F/dt - div(k_F/mu grad p_F) + sigma* k_f/mu (p_F - p_f)
            q_f = phiC_f dp_f/dt - div(k_f/mu grad p_f) + sigma* k_f/mu (p_f - p_F)
                                                    + sigma k_m/mu (p_f - p_m)
            q_m = phiC_m dp_m/dt - div(k_m/mu grad p_m) + sigma k_m/mu (p_m - p_f)
The exact fields need not satisfy the interface conditions of Sec. 2, so their defects on
Gamma (y = 1, n_c = (0,-1), n_p = (0,1), tau = (1,0)) are carried as interface data:
  g_N = -n_c.T n_c - p_F/rho
  g_T = -tau.(T n_c) - (alpha nu / sqrt(k_F)) tau.(u + k_F/mu grad p_F)
  g_F = u.n_c - k_F/mu grad p_F . n_p,   g_f = -k_f/mu grad p_f . n_p,
  g_m = -k_m/mu grad p_m . n_p
They enter the weak forms as  -eta<g_N, v.n_c> - eta<g_T, v.tau>  (conduit) and
-<g_i, v_i> (porous); with them the exact fields satisfy the weak problem of Sec. 3.1.
"""
import numpy as np
import sympy as sp

X, Y, T = sp.symbols("x y t", real=True)


def _fields(mms_id):
    pi = sp.pi
    if mms_id == 1:
        e = sp.exp(-T)
        u = (sp.sin(pi * X) * sp.cos(pi * Y) * e, -sp.cos(pi * X) * sp.sin(pi * Y) * e)
        p = sp.cos(pi * X) * sp.cos(pi * Y) * e
        base = sp.cos(pi * X) * sp.cos(pi * Y) * e
        pd = (3 * base, 2 * base, 1 * base)            # F, f, m
        return u, p, pd
    if mms_id == 3:
        u = (X ** 2, -2 * X * Y)
        p = X + Y
        r2 = X ** 2 + Y ** 2
        pd = (3 * r2, 2 * r2, 1 * r2)
        return u, p, pd
    if mms_id == 0:
        z = sp.Integer(0)
        return (z, z), z, (z, z, z)
    raise ValueError(f"unknown manufactured solution {mms_id}")


def _lam(expr):
    f = sp.lambdify((X, Y, T), expr, "numpy")

    def g(x, y, t):
        x = np.asarray(x, dtype=float)
        y = np.asarray(y, dtype=float)
        return np.broadcast_to(np.asarray(f(x, y, t), dtype=float), np.broadcast(x, y).shape).copy()
    return g


class MMS:
    def __init__(self, mms_id, prm):
        u, p, pd = _fields(mms_id)
        nu, mu, rho, al = (sp.nsimplify(v) if False else sp.Float(v, 30)
                           for v in (prm.nu, prm.mu, prm.rho, prm.alpha))
        sig, sigs = sp.Float(prm.sigma, 30), sp.Float(prm.sigma_star, 30)
        k = [sp.Float(v, 30) for v in prm.k]
        phiC = [sp.Float(v, 30) for v in prm.phiC]
        ux, uy = u
        grad = lambda s: (sp.diff(s, X), sp.diff(s, Y))
        lap = lambda s: sp.diff(s, X, 2) + sp.diff(s, Y, 2)
        divu = sp.diff(ux, X) + sp.diff(uy, Y)
        # -div(2 nu D(u)) = -nu (lap u + grad div u)
        f = []
        for a, ua in enumerate(u):
            conv = ux * sp.diff(ua, X) + uy * sp.diff(ua, Y)
            f.append(sp.diff(ua, T) - nu * (lap(ua) + grad(divu)[a]) + grad(p)[a] + conv)
        pF, pf, pm = pd
        cFf = sigs * k[1] / mu
        cfm = sig * k[2] / mu
        q = [phiC[0] * sp.diff(pF, T) - k[0] / mu * lap(pF) + cFf * (pF - pf),
             phiC[1] * sp.diff(pf, T) - k[1] / mu * lap(pf) + cFf * (pf - pF) + cfm * (pf - pm),
             phiC[2] * sp.diff(pm, T) - k[2] / mu * lap(pm) + cfm * (pm - pf)]
        # stress and interface defects on y = 1
        gu = [[sp.diff(ux, X), sp.diff(ux, Y)], [sp.diff(uy, X), sp.diff(uy, Y)]]
        Tm = [[nu * (gu[a][c] + gu[c][a]) - (p if a == c else 0) for c in range(2)] for a in range(2)]
        n_c = (0, -1)
        n_p = (0, 1)
        tau = (1, 0)
        Tn = [sum(Tm[a][c] * n_c[c] for c in range(2)) for a in range(2)]
        nTn = sum(n_c[a] * Tn[a] for a in range(2))
        gN = -nTn - pF / rho
        gradpF = grad(pF)
        gT = (-sum(tau[a] * Tn[a] for a in range(2))
              - al * nu / sp.sqrt(k[0]) * sum(tau[a] * (u[a] + k[0] / mu * gradpF[a]) for a in range(2)))
        g1 = sum(u[a] * n_c[a] for a in range(2)) - k[0] / mu * sum(gradpF[a] * n_p[a] for a in range(2))
        gf = -k[1] / mu * sum(grad(pf)[a] * n_p[a] for a in range(2))
        gm = -k[2] / mu * sum(grad(pm)[a] * n_p[a] for a in range(2))
        on_gamma = lambda e: e.subs(Y, 1)
        self._gu = [[_lam(sp.diff(ua, v)) for v in (X, Y)] for ua in u]
        self._gpd = [[_lam(sp.diff(e, v)) for v in (X, Y)] for e in pd]
        self._u = [_lam(e) for e in u]
        self._p = _lam(p)
        self._pd = [_lam(e) for e in pd]
        self._f = [_lam(sp.simplify(e)) for e in f]
        self._q = [_lam(sp.simplify(e)) for e in q]
        self._gN = _lam(on_gamma(gN))
        self._gT = _lam(on_gamma(gT))
        self._gd = [_lam(on_gamma(g1)), _lam(on_gamma(gf)), _lam(on_gamma(gm))]
        self.steady = mms_id in (0, 3)

    # exact fields
    def u(self, x, y, t):
        return np.stack([g(x, y, t) for g in self._u], axis=-1)

    def grad_u(self, x, y, t):
        return np.stack([np.stack([g(x, y, t) for g in row], axis=-1) for row in self._gu], axis=-2)

    def grad_pd(self, i, x, y, t):
        return np.stack([g(x, y, t) for g in self._gpd[i]], axis=-1)

    def p(self, x, y, t):
        return self._p(x, y, t)

    def pd(self, i, x, y, t):
        return self._pd[i](x, y, t)

    # data
    def f(self, x, y, t):
        return np.stack([g(x, y, t) for g in self._f], axis=-1)

    def q(self, i, x, y, t):
        return self._q[i](x, y, t)

    def gN(self, x, t):
        return self._gN(x, np.ones_like(x), t)

    def gT(self, x, t):
        return self._gT(x, np.ones_like(x), t)

    def gd(self, i, x, t):
        return self._gd[i](x, np.ones_like(x), t)
