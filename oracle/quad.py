"""Quadrature rules used by the oracle.

Cells: the symmetric 7-point rule of degree 5 on the reference triangle
{(x, y): x, y >= 0, x + y <= 1} (Radon's rule, as tabulated by Stroud).  Its points and
weights have closed forms in sqrt(15).  Degree 5 integrates every bilinear and trilinear
integrand of the P2-P1 weak forms of Sec. 3.1 exactly (the convection term
((w.grad)u, v) with w, u, v in P2 has degree 5).

Edges: Gauss-Legendre with 3 points on [0, 1] (degree 5), taken from NumPy.
"""
import numpy as np


def triangle_rule7():
    """Return (points (7,2), weights (7,)) on the reference triangle; weights sum to 1/2."""
    s = np.sqrt(15.0)
    a1 = (6.0 - s) / 21.0
    a2 = (6.0 + s) / 21.0
    w1 = (155.0 - s) / 2400.0
    w2 = (155.0 + s) / 2400.0
    pts = [(1.0 / 3.0, 1.0 / 3.0),
           (a1, a1), (1.0 - 2.0 * a1, a1), (a1, 1.0 - 2.0 * a1),
           (a2, a2), (1.0 - 2.0 * a2, a2), (a2, 1.0 - 2.0 * a2)]
    wts = [9.0 / 80.0, w1, w1, w1, w2, w2, w2]
    return np.array(pts), np.array(wts)


def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule mapped to [0, 1] (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def duffy_rule(nu, nv):
    """Collapsed (Duffy) tensor rule on the reference triangle: x = u, y = v (1 - u),
    dA = (1 - u) du dv.  Used only by tests as an independent cross-check."""
    u, wu = gauss_legendre_01(nu)
    v, wv = gauss_legendre_01(nv)
    U, V = np.meshgrid(u, v, indexing="ij")
    W = np.outer(wu, wv) * (1.0 - U)
    return np.stack([U.ravel(), (V * (1.0 - U)).ravel()], axis=1), W.ravel()
