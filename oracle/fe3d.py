"""P2 / P1 Lagrange elements on tetrahedra, the quadrature that integrates the weak forms
of Sec. 3.1 exactly in 3D, and their element integrals (forms a_F, a_f, a_m, a_{c eta},
b_{N eta}, b_eta and the Gamma forms on triangular faces).

Test infrastructure (see the package docstring).

Cells: the collapsed (Duffy / conical product) rule on the reference tetrahedron
{xi, eta, zeta >= 0, xi + eta + zeta <= 1}: x = u, y = v (1 - u), z = w (1 - u)(1 - v),
dV = (1-u)^2 (1-v) du dv dw, with 3-point Gauss-Jacobi rules for the weights (1-u)^2 and
(1-v) and 3-point Gauss-Legendre in w (SciPy's roots_jacobi / NumPy's leggauss): a
polynomial of total degree <= 5 becomes one of degree <= 5 in each of u, v, w, which the
3-point rules integrate exactly.  27 points; degree 5 covers the convection term
((w.grad)u, v) with w, u, v in P2.
Faces: the 7-point degree-5 triangle rule of ``quad``.

Vectorised over elements: coordinates X have shape (ne, 4, 3).
"""
import numpy as np
from scipy.special import roots_jacobi

from .quad import triangle_rule7


def tet_rule():
    """(points (27, 3), weights (27,)) on the reference tetrahedron; weights sum to 1/6."""
    def gj(n, alpha):
        x, w = roots_jacobi(n, alpha, 0.0)          # weight (1-x)^alpha on [-1, 1]
        return 0.5 * (x + 1.0), w / 2.0 ** (alpha + 1)
    u, wu = gj(3, 2.0)
    v, wv = gj(3, 1.0)
    s, ws = gj(3, 0.0)
    pts, wts = [], []
    for a in range(3):
        for b in range(3):
            for c in range(3):
                x = u[a]
                y = v[b] * (1.0 - u[a])
                z = s[c] * (1.0 - u[a]) * (1.0 - v[b])
                pts.append((x, y, z))
                wts.append(wu[a] * wv[b] * ws[c])
    return np.array(pts), np.array(wts)


QP, QW = tet_rule()
EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
DLAM = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def p2_basis(pts):
    """Values (nq, 10) and reference gradients (nq, 10, 3) of the P2 basis at points:
    vertices lambda_i (2 lambda_i - 1), then edges 4 lambda_a lambda_b in EDGES order."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    L = np.stack([1.0 - x - y - z, x, y, z], axis=1)
    N = np.zeros((len(x), 10))
    dN = np.zeros((len(x), 10, 3))
    for i in range(4):
        N[:, i] = L[:, i] * (2 * L[:, i] - 1)
        dN[:, i, :] = (4 * L[:, i] - 1)[:, None] * DLAM[i]
    for k, (a, b) in enumerate(EDGES):
        N[:, 4 + k] = 4 * L[:, a] * L[:, b]
        dN[:, 4 + k, :] = 4 * (L[:, a][:, None] * DLAM[b] + L[:, b][:, None] * DLAM[a])
    return N, dN


def p1_basis(pts):
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    N = np.stack([1.0 - x - y - z, x, y, z], axis=1)
    dN = np.broadcast_to(DLAM, (len(x), 4, 3))
    return N, dN


PHI, DPHI = p2_basis(QP)        # (27,10), (27,10,3)
PSI, DPSI = p1_basis(QP)        # (27,4), (27,4,3)


def geometry(X):
    """Affine map x = a + J xi.  Returns detJ (ne,), Jinv (ne,3,3), quadrature points in
    physical space (ne, nq, 3) and weights W = w_q |detJ| (ne, nq)."""
    a = X[:, 0, :]
    J = np.stack([X[:, 1, :] - a, X[:, 2, :] - a, X[:, 3, :] - a], axis=2)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    xq = a[:, None, :] + np.einsum("ecr,qr->eqc", J, QP)
    W = np.abs(det)[:, None] * QW[None, :]
    return det, Jinv, xq, W


def grads(Jinv, dref):
    """Physical gradients (ne, nq, nb, 3) from reference gradients (nq, nb, 3)."""
    return np.einsum("qir,erc->eqic", dref, Jinv)


def mass_p2(W):
    return np.einsum("eq,qi,qj->eij", W, PHI, PHI)


def stiff_p2(W, G):
    return np.einsum("eq,eqic,eqjc->eij", W, G, G)


def load_p2(W, fq):
    return np.einsum("eq,eq,qi->ei", W, fq, PHI)


def at_qp(vals):
    if vals.ndim == 2:
        return np.einsum("qi,ei->eq", PHI, vals)
    return np.einsum("qi,eid->eqd", PHI, vals)


def grad_at_qp(G, vals):
    if vals.ndim == 2:
        return np.einsum("eqic,ei->eqc", G, vals)
    return np.einsum("eqic,eid->eqdc", G, vals)


def oseen_blocks(W, G, w, Gw, dt, prm):
    """Element blocks of the local conduit operator (Alg. 3 Step 3(2)) in 3D:
        eta/dt (e, v) + 2 nu eta (D(e), D(v)) + b_N(e, w, v) + b_N(w, e, v) + b(v, delta)
    and the pressure rows -b(e, q).  w at qp (ne,nq,3), Gw[..., a, c] = d w_a / d x_c.
    Returns Kvv (ne,10,3,10,3) [test i,a ; trial j,b], Kvp (ne,10,3,4), Kpv (ne,4,10,3)."""
    eta, nu = prm.eta, prm.nu
    I3 = np.eye(3)
    M = np.einsum("eq,qi,qj->eij", W, PHI, PHI)
    S = np.einsum("eq,eqic,eqjc->eij", W, G, G)
    C = np.einsum("eq,eqia,eqjb->eiajb", W, G, G)
    Kvv = (eta / dt) * np.einsum("eij,ab->eiajb", M, I3)
    Kvv += nu * eta * (np.einsum("eij,ab->eiajb", S, I3) + np.einsum("ejaib->eiajb", C))
    Kvv += eta * np.einsum("eq,qi,qj,eqab->eiajb", W, PHI, PHI, Gw)
    conv = np.einsum("eq,qi,eqc,eqjc->eij", W, PHI, w, G)
    Kvv += eta * np.einsum("eij,ab->eiajb", conv, I3)
    Kvp = -eta * np.einsum("eq,qk,eqia->eiak", W, PSI, G)
    Kpv = eta * np.einsum("eq,qk,eqjb->ekjb", W, PSI, G)
    return Kvv, Kvp, Kpv


def ns_residual_volume(W, G, u, un, Gu, p, f, dt, prm):
    """Volume part of the conduit residual (3D):
        eta/dt (u - un, v) + 2 nu eta (D(u), D(v)) + b_N(u, u, v) + b(v, p) - eta (f, v)
    and pressure rows eta (q, div u).  Returns Rv (ne,10,3), Rp (ne,4)."""
    eta, nu = prm.eta, prm.nu
    Rv = (eta / dt) * np.einsum("eq,qi,eqa->eia", W, PHI, u - un)
    Du = 0.5 * (Gu + np.swapaxes(Gu, 2, 3))
    Rv += 2.0 * nu * eta * np.einsum("eq,eqac,eqic->eia", W, Du, G)
    conv = np.einsum("eqc,eqac->eqa", u, Gu)
    Rv += eta * np.einsum("eq,qi,eqa->eia", W, PHI, conv)
    Rv += -eta * np.einsum("eq,eq,eqia->eia", W, p, G)
    Rv += -eta * np.einsum("eq,qi,eqa->eia", W, PHI, f)
    divu = np.einsum("eqaa->eq", Gu)
    Rp = eta * np.einsum("eq,qk,eq->ek", W, PSI, divu)
    return Rv, Rp


# ---------------------------------------------------------------- faces on Gamma
FQ, FW = triangle_rule7()
FEDGES = [(0, 1), (0, 2), (1, 2)]


def p2_face_basis(pts):
    """P2 basis on a triangle, nodes (v0, v1, v2, m01, m02, m12): values (nq,6) and
    reference gradients (nq,6,2)."""
    x, y = pts[:, 0], pts[:, 1]
    L = np.stack([1.0 - x - y, x, y], axis=1)
    dl = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    N = np.zeros((len(x), 6))
    dN = np.zeros((len(x), 6, 2))
    for i in range(3):
        N[:, i] = L[:, i] * (2 * L[:, i] - 1)
        dN[:, i, :] = (4 * L[:, i] - 1)[:, None] * dl[i]
    for k, (a, b) in enumerate(FEDGES):
        N[:, 3 + k] = 4 * L[:, a] * L[:, b]
        dN[:, 3 + k, :] = 4 * (L[:, a][:, None] * dl[b] + L[:, b][:, None] * dl[a])
    return N, dN


FPHI, FDPHI = p2_face_basis(FQ)


def face_geometry(P):
    """Faces in the plane z = const given by the (x, y) of their three vertices (nf, 3, 2).
    Returns area weights (nf, 7), quadrature points (nf, 7, 2) and the inverse Jacobians
    (nf, 2, 2) of the in-plane affine maps."""
    a = P[:, 0, :]
    J = np.stack([P[:, 1, :] - a, P[:, 2, :] - a], axis=2)
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.linalg.inv(J)
    xq = a[:, None, :] + np.einsum("ecr,qr->eqc", J, FQ)
    W = np.abs(det)[:, None] * FW[None, :]
    return W, xq, Jinv
