"""P2 / P1 Lagrange elements on triangles and element integrals of the weak forms of
Sec. 3.1 (forms a_F, a_f, a_m, a_{c eta}, b_{N eta}, b_eta and the Gamma forms), all by
quadrature with the degree-5 rule of ``quad``.

Vectorised over elements: coordinates X have shape (ne, 3, 2).
"""
import numpy as np

from .quad import triangle_rule7, gauss_legendre_01

QP, QW = triangle_rule7()


def p2_basis(pts):
    """Values (nq, 6) and reference gradients (nq, 6, 2) of the P2 basis at points."""
    x, y = pts[:, 0], pts[:, 1]
    l0, l1, l2 = 1.0 - x - y, x, y
    N = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                  4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=1)
    # d lambda / d(x, y): l0 -> (-1,-1), l1 -> (1,0), l2 -> (0,1)
    dl = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    L = np.stack([l0, l1, l2], axis=1)
    dN = np.zeros((len(x), 6, 2))
    for i in range(3):
        dN[:, i, :] = (4 * L[:, i] - 1)[:, None] * dl[i]
    pairs = [(0, 1), (1, 2), (2, 0)]
    for k, (a, b) in enumerate(pairs):
        dN[:, 3 + k, :] = 4 * (L[:, a][:, None] * dl[b] + L[:, b][:, None] * dl[a])
    return N, dN


def p1_basis(pts):
    x, y = pts[:, 0], pts[:, 1]
    N = np.stack([1.0 - x - y, x, y], axis=1)
    dN = np.broadcast_to(np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]]), (len(x), 3, 2))
    return N, dN


PHI, DPHI = p2_basis(QP)        # (7,6), (7,6,2)
PSI, DPSI = p1_basis(QP)        # (7,3), (7,3,2)


def geometry(X):
    """Affine map x = a + J xi.  Returns detJ (ne,), Jinv (ne,2,2), quadrature points
    in physical space (ne, nq, 2) and weights W = w_q |detJ| (ne, nq)."""
    a = X[:, 0, :]
    J = np.stack([X[:, 1, :] - a, X[:, 2, :] - a], axis=2)     # columns b-a, c-a
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.empty_like(J)
    Jinv[:, 0, 0] = J[:, 1, 1] / det
    Jinv[:, 1, 1] = J[:, 0, 0] / det
    Jinv[:, 0, 1] = -J[:, 0, 1] / det
    Jinv[:, 1, 0] = -J[:, 1, 0] / det
    xq = a[:, None, :] + np.einsum("ecr,qr->eqc", J, QP)
    W = np.abs(det)[:, None] * QW[None, :]
    return det, Jinv, xq, W


def grads(Jinv, dref):
    """Physical gradients (ne, nq, nb, 2) from reference gradients (nq, nb, 2)."""
    return np.einsum("qir,erc->eqic", dref, Jinv)


# ---------------------------------------------------------------- scalar P2 forms
def mass_p2(W):
    return np.einsum("eq,qi,qj->eij", W, PHI, PHI)


def stiff_p2(W, G):
    return np.einsum("eq,eqic,eqjc->eij", W, G, G)


def load_p2(W, fq):
    """(f, phi_i) with f given at quadrature points (ne, nq)."""
    return np.einsum("eq,eq,qi->ei", W, fq, PHI)


def at_qp(vals):
    """Values at quadrature points of a P2 field given at element nodes (ne, 6[, d])."""
    if vals.ndim == 2:
        return np.einsum("qi,ei->eq", PHI, vals)
    return np.einsum("qi,eid->eqd", PHI, vals)


def grad_at_qp(G, vals):
    """Gradient at quadrature points: (ne, nq, 2) for scalar, (ne, nq, d, 2) for vector."""
    if vals.ndim == 2:
        return np.einsum("eqic,ei->eqc", G, vals)
    return np.einsum("eqic,eid->eqdc", G, vals)


# ---------------------------------------------------------------- Oseen / NS forms
def oseen_blocks(W, G, GP, w, Gw, dt, prm):
    """Element blocks of the operator of the local conduit problem (Alg. 3 Step 3(2)):
        eta/dt (e, v) + 2 nu eta (D(e), D(v)) + b_N(e, w, v) + b_N(w, e, v) + b(v, delta)
    and the pressure rows -b(e, q).  w: linearisation velocity at qp (ne,nq,2),
    Gw = grad w at qp (ne,nq,2,2) with Gw[...,a,c] = d w_a / d x_c.
    Returns Kvv (ne,6,2,6,2) [test i,a ; trial j,b], Kvp (ne,6,2,3), Kpv (ne,3,6,2).
    (The Beavers-Joseph-Saffman Gamma term is added separately.)"""
    eta, nu = prm.eta, prm.nu
    M = np.einsum("eq,qi,qj->eij", W, PHI, PHI)
    S = np.einsum("eq,eqic,eqjc->eij", W, G, G)                       # grad phi_i . grad phi_j
    C = np.einsum("eq,eqia,eqjb->eiajb", W, G, G)                     # d_a phi_i d_b phi_j
    I2 = np.eye(2)
    Kvv = (eta / dt) * np.einsum("eij,ab->eiajb", M, I2)
    # 2 nu eta D(phi_j e_b):D(phi_i e_a) = nu eta (delta_ab grad.grad + d_a phi_j d_b phi_i)
    Kvv += nu * eta * (np.einsum("eij,ab->eiajb", S, I2) + np.einsum("ejaib->eiajb", C))
    # b_N(e, w, v) = eta ((e . grad) w, v): trial phi_j e_b, test phi_i e_a -> phi_j d_b w_a phi_i
    Kvv += eta * np.einsum("eq,qi,qj,eqab->eiajb", W, PHI, PHI, Gw)
    # b_N(w, e, v) = eta ((w . grad) e, v) -> delta_ab (w . grad phi_j) phi_i
    conv = np.einsum("eq,qi,eqc,eqjc->eij", W, PHI, w, G)
    Kvv += eta * np.einsum("eij,ab->eiajb", conv, I2)
    # b(v, delta) = -eta (delta, div v): test phi_i e_a, trial psi_k
    Kvp = -eta * np.einsum("eq,qk,eqia->eiak", W, PSI, G)
    # pressure rows: -b(e, q) = eta (q, div e)
    Kpv = eta * np.einsum("eq,qk,eqjb->ekjb", W, PSI, G)
    return Kvv, Kvp, Kpv


def ns_residual_volume(W, G, u, un, Gu, p, f, dt, prm):
    """Volume part of the conduit residual for trial state (u, p) at qp, previous velocity
    un at qp and forcing f at qp:
        eta/dt (u - un, v) + 2 nu eta (D(u), D(v)) + b_N(u, u, v) + b(v, p) - eta (f, v)
    and pressure rows -b(u, q) = eta (q, div u).  Returns Rv (ne,6,2), Rp (ne,3)."""
    eta, nu = prm.eta, prm.nu
    Rv = (eta / dt) * np.einsum("eq,qi,eqa->eia", W, PHI, u - un)
    Du = 0.5 * (Gu + np.swapaxes(Gu, 2, 3))                                  # D(u)_{ac}
    # 2 nu eta D(u):D(phi_i e_a) = 2 nu eta sum_c D(u)_{ac} d_c phi_i
    Rv += 2.0 * nu * eta * np.einsum("eq,eqac,eqic->eia", W, Du, G)
    conv = np.einsum("eqc,eqac->eqa", u, Gu)                                  # (u.grad)u
    Rv += eta * np.einsum("eq,qi,eqa->eia", W, PHI, conv)
    Rv += -eta * np.einsum("eq,eq,eqia->eia", W, p, G)                       # -eta (p, div v)
    Rv += -eta * np.einsum("eq,qi,eqa->eia", W, PHI, f)
    divu = np.einsum("eqaa->eq", Gu)
    Rp = eta * np.einsum("eq,qk,eq->ek", W, PSI, divu)
    return Rv, Rp


# ---------------------------------------------------------------- edges on Gamma
EQ, EW = gauss_legendre_01(3)


def p2_edge_basis(s):
    """1D P2 basis on an edge parameterised by s in [0,1]; nodes (s=0, s=1, s=1/2)."""
    return np.stack([(1 - s) * (1 - 2 * s), s * (2 * s - 1), 4 * s * (1 - s)], axis=1)


def p2_edge_dbasis(s):
    return np.stack([4 * s - 3, 4 * s - 1, 4 - 8 * s], axis=1)


EPHI = p2_edge_basis(EQ)        # (3 qp, 3 nodes)
EDPHI = p2_edge_dbasis(EQ)


def edge_mass(length):
    """int_e phi_i phi_j for P2 edge basis, (ned, 3, 3)."""
    return np.einsum("q,qi,qj,e->eij", EW, EPHI, EPHI, length)
