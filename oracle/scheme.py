"""Algorithm 3 of the paper (local parallel two-grid finite element method, Sec. 5),
written out plainly in FP64 with NumPy/SciPy.

Per time step n -> n+1 (t = (n+1) dt):
  Step 1 (coarse, eqs. pFFully, pfFully, pmFully): three decoupled P2 Darcy solves on T_H
         with the partner pressures and the conduit velocity on Gamma lagged at t_n;
         (eq. pcFully): the nonlinear conduit problem on T_H with p_FH^n on Gamma, solved by
         Newton's method (||delta||/||x|| <= 1e-14 or 30 iterations).
  Step 2: the overlapping subdomains Omega_j (``mesh.make_subdomains``).
  Step 3 (eqs. pFlocalFully, pflocalFully, pmlocalFully, uclocalFully): on every Omega_j a
         fine correction whose right-hand side is the fine residual of the coarse solution
         plus the lagged local corrections e_j^n.
  Step 4: correction of data on D_j; shared closure nodes are averaged (weights
         1 / #{j : x in closure(D_j)}).
Coarse functions are represented on the fine mesh by their fine nodal interpolant I_h
(exact when T_h is nested in T_H).  Readings of points the paper leaves open: homogeneous
Dirichlet correction on the artificial boundary, e = I_h g - I_h I_H g on the global
Dirichlet boundary, natural conditions on Gamma, local corrections in the compactly supported spaces
X_c0^h x Q_0^h of Sec. 3.2 (velocity and pressure corrections vanish on the artificial
boundary), nodal interpolation for the initial data.
The linear solves use SciPy's sparse LU (SuperLU) -- a library primitive independent of
the GPU library's band factorisations.
"""
import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import fe
from .mesh import Mesh2D, region_breaks, make_subdomains
from .mms import MMS

FIELDS = ("ux", "uy", "p", "pF", "pf", "pm")


# ---------------------------------------------------------------------------- helpers
def prolongation(mH, mh, kind):
    """Sparse matrix of the fine nodal interpolant of coarse P2 (kind='p2') or P1 ('p1')
    functions: row = fine node (P2 node or vertex), column = coarse node."""
    pts = mh.node if kind == "p2" else mh.vert
    nb = 6 if kind == "p2" else 3
    ci = np.clip(np.searchsorted(mH.xs, pts[:, 0], side="right") - 1, 0, mH.nx - 1)
    cj = np.clip(np.searchsorted(mH.ys, pts[:, 1], side="right") - 1, 0, mH.ny - 1)
    rows, cols, vals = [], [], []
    for t in (0, 1):
        tri = 2 * (ci + mH.nx * cj) + t
        X = mH.vert[mH.tri[tri]]
        det, Jinv, _, _ = fe.geometry(X)
        xi = np.einsum("erc,ec->er", Jinv, pts - X[:, 0, :])
        lam = np.stack([1 - xi[:, 0] - xi[:, 1], xi[:, 0], xi[:, 1]], axis=1)
        inside = lam.min(axis=1) >= -1e-12
        if t == 1:
            inside &= ~taken
        taken = inside if t == 0 else taken | inside
        idx = np.nonzero(inside)[0]
        if kind == "p2":
            N, _ = fe.p2_basis(xi[idx])
            nodes = mH.tri6[tri[idx]]
        else:
            N, _ = fe.p1_basis(xi[idx])
            nodes = mH.tri[tri[idx]]
        rows.append(np.repeat(idx, nb))
        cols.append(nodes.ravel())
        vals.append(N.ravel())
    assert taken.all()
    n_c = mH.nn if kind == "p2" else mH.nv
    P = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(len(pts), n_c))
    P.data[np.abs(P.data) < 1e-15] = 0.0
    P.eliminate_zeros()
    return P


def coo_assemble(dofs_r, dofs_c, vals, n):
    r = np.broadcast_to(dofs_r, vals.shape).ravel()
    c = np.broadcast_to(dofs_c, vals.shape).ravel()
    return sps.csr_matrix((vals.ravel(), (r, c)), shape=(n, n))


def vec_assemble(dofs, vals, n):
    out = np.zeros(n)
    np.add.at(out, dofs.ravel(), vals.ravel())
    return out


class Region:
    """Geometry, element data and Gamma edges of one region mesh (or of one subdomain)."""

    def __init__(self, mesh, tris, tri6, tri3, nn, nv, gamma_edges, gnode):
        self.mesh = mesh
        X = mesh.tri_coords(tris)
        self.det, self.Jinv, self.xq, self.W = fe.geometry(X)
        self.G = fe.grads(self.Jinv, fe.DPHI)
        self.tri6, self.tri3, self.nn, self.nv = tri6, tri3, nn, nv
        self.gamma_edges = gamma_edges
        self.gnode = gnode                                  # local P2 node -> global node
        nodes = mesh.node[gnode]
        self.xy = nodes
        if len(gamma_edges):
            xa = nodes[gamma_edges[:, 0], 0]
            xb = nodes[gamma_edges[:, 1], 0]
            self.elen = np.abs(xb - xa)
            s = fe.EQ
            self.exq = xa[:, None] + (xb - xa)[:, None] * s[None, :]     # (ned, 3)
            self.ew = np.abs(xb - xa)[:, None] * fe.EW[None, :]
            # the P2 edge basis is ordered (left vertex, right vertex, midpoint)
            self.edge_nodes = gamma_edges
        else:
            self.elen = np.zeros(0)
            self.edge_nodes = np.zeros((0, 3), dtype=np.int64)

    # ---- Gamma integrals on edges (tau = +x); values given at the 3 edge nodes
    def gamma_mass(self):
        return fe.edge_mass(self.elen)

    def gamma_load(self, gq):
        """int_Gamma g phi_i for g given at edge quadrature points (ned, 3)."""
        return np.einsum("eq,eq,qi->ei", self.ew, gq, fe.EPHI)

    def gamma_trace_qp(self, nodal):
        return np.einsum("qi,ei->eq", fe.EPHI, nodal[self.edge_nodes])

    def gamma_dtau_qp(self, nodal):
        d = np.einsum("qi,ei->eq", fe.EDPHI, nodal[self.edge_nodes])
        return d / self.elen[:, None]


def region_whole(mesh, region):
    gamma_J = 0 if region == "c" else 2 * mesh.ny
    row = mesh.half[gamma_J, :]
    ge = np.stack([row[0:-1:2], row[2::2], row[1::2]], axis=1)
    return Region(mesh, np.arange(len(mesh.tri)), mesh.tri6, mesh.tri, mesh.nn, mesh.nv, ge,
                  np.arange(mesh.nn))


def region_sub(mesh, sub):
    return Region(mesh, sub.tris, sub.tri6, sub.tri3, len(sub.gnode), len(sub.vloc),
                  sub.gamma_edges, sub.gnode)


# ---------------------------------------------------------------------------- operators
class Ops:
    """Element-level operators of Sec. 3.1 on a Region, with the scheme's coefficients."""

    def __init__(self, R, prm, dt):
        self.R, self.prm, self.dt = R, prm, dt
        self.M = fe.mass_p2(R.W)
        self.K = fe.stiff_p2(R.W, R.G)
        nn, nv = R.nn, R.nv
        self.vdof = 2 * R.tri6[:, :, None] + np.arange(2)[None, None, :]     # (ne,6,2)
        self.pdof = 2 * nn + R.tri3                                          # (ne,3)
        self.nvel = 2 * nn
        self.ntot = 2 * nn + nv

    # -- Darcy (eqs. pFlocalFully..pmlocalFully): A_i = (phiC_i/dt + c_i) M + k_i/mu K
    def darcy_coeffs(self):
        p = self.prm
        kF, kf, km = p.k
        cF = p.sigma_star * kf / p.mu
        cf = (p.sigma * km + p.sigma_star * kf) / p.mu
        cm = p.sigma * km / p.mu
        return [(p.phiC[0] / self.dt + cF, kF / p.mu), (p.phiC[1] / self.dt + cf, kf / p.mu),
                (p.phiC[2] / self.dt + cm, km / p.mu)]

    def darcy_matrix(self, i):
        a, b = self.darcy_coeffs()[i]
        vals = a * self.M + b * self.K
        d = self.R.tri6
        return coo_assemble(d[:, :, None], d[:, None, :], vals, self.R.nn)

    def mass_matrix(self):
        d = self.R.tri6
        return coo_assemble(d[:, :, None], d[:, None, :], self.M, self.R.nn)

    def darcy_load(self, q_at_qp):
        return vec_assemble(self.R.tri6, fe.load_p2(self.R.W, q_at_qp), self.R.nn)

    def gamma_vec(self, edge_vals):
        return vec_assemble(self.R.edge_nodes, edge_vals, self.R.nn)

    # -- conduit
    def oseen_matrix(self, w_nodal):
        """Jacobian of the conduit residual about velocity w (nodal (nn,2)), incl. BJS."""
        R, prm = self.R, self.prm
        we = w_nodal[R.tri6]
        wq = fe.at_qp(we)
        Gw = fe.grad_at_qp(R.G, we)
        Kvv, Kvp, Kpv = fe.oseen_blocks(R.W, R.G, None, wq, Gw, self.dt, prm)
        n = self.ntot
        A = coo_assemble(self.vdof[:, :, :, None, None], self.vdof[:, None, None, :, :], Kvv, n)
        A = A + coo_assemble(self.vdof[:, :, :, None], self.pdof[:, None, None, :], Kvp, n)
        A = A + coo_assemble(self.pdof[:, :, None, None], self.vdof[:, None, :, :], Kpv, n)
        if len(R.edge_nodes):
            bjs = prm.eta * prm.nu * prm.alpha / np.sqrt(prm.k[0])
            Me = R.gamma_mass() * bjs
            dx = 2 * R.edge_nodes                                  # x-components (tau = e_x)
            A = A + coo_assemble(dx[:, :, None], dx[:, None, :], Me, n)
        return A.tocsr()

    def ns_residual(self, u, un, p, t, mms, pF_gamma):
        """Conduit residual of eq. uclocalFully's bracket / eq. pcFully:
           eta/dt(u-un,v) + a_c(u,v) + b(v,p) - b(u,q) + b_N(u,u,v)
           + eta/rho <pF, v.n_c> + eta nu alpha sqrt(kF)/mu <d_tau pF, v.tau>
           - eta (f, v) + eta <g_N, v.n_c> + eta <g_T, v.tau>.
        u, un nodal (nn,2); p at vertices (nv,); pF_gamma nodal porous pressure on the
        Gamma nodes of this region (array over local nodes, used on Gamma only)."""
        R, prm = self.R, self.prm
        ue, une = u[R.tri6], un[R.tri6]
        uq, unq = fe.at_qp(ue), fe.at_qp(une)
        Gu = fe.grad_at_qp(R.G, ue)
        pq = np.einsum("qk,ek->eq", fe.PSI, p[R.tri3])
        fq = mms.f(R.xq[..., 0], R.xq[..., 1], t)
        Rv, Rp = fe.ns_residual_volume(R.W, R.G, uq, unq, Gu, pq, fq, self.dt, prm)
        r = np.zeros(self.ntot)
        np.add.at(r, self.vdof.ravel(), Rv.ravel())
        np.add.at(r, self.pdof.ravel(), Rp.ravel())
        if len(R.edge_nodes):
            eta, nu, al, kF, mu, rho = prm.eta, prm.nu, prm.alpha, prm.k[0], prm.mu, prm.rho
            bjs = eta * nu * al / np.sqrt(kF)
            Me = R.gamma_mass()
            ux_e = u[R.edge_nodes, 0]
            rx = bjs * np.einsum("eij,ej->ei", Me, ux_e)                   # BJS: <u.tau, v.tau>
            pFq = R.gamma_trace_qp(pF_gamma)
            dpFq = R.gamma_dtau_qp(pF_gamma)
            xq = R.exq
            gN = mms.gN(xq, t)
            gT = mms.gT(xq, t)
            # v.n_c = -v_y on Gamma (n_c = (0,-1)); v.tau = v_x
            ry = -(eta / rho) * R.gamma_load(pFq) - eta * R.gamma_load(gN)
            rx = rx + (eta * nu * al * np.sqrt(kF) / mu) * R.gamma_load(dpFq) + eta * R.gamma_load(gT)
            np.add.at(r, (2 * R.edge_nodes).ravel(), rx.ravel())
            np.add.at(r, (2 * R.edge_nodes + 1).ravel(), ry.ravel())
        return r

    def mass_vec(self, nodal_vec):
        """(w, v) for a nodal vector field w -> velocity-dof vector."""
        R = self.R
        vals = np.einsum("eij,eja->eia", self.M, nodal_vec[R.tri6])
        r = np.zeros(self.ntot)
        np.add.at(r, self.vdof.ravel(), vals.ravel())
        return r


def solve_sparse(A, b):
    lu = spla.splu(sps.csc_matrix(A))
    return lu.solve(b)


# ---------------------------------------------------------------------------- the oracle
class TwoGridOracle:
    """Algorithm 3 on a 2D workload (see ``workloads``)."""

    def __init__(self, w, coarse_only=False):
        self.w, self.prm, self.dt = w, w.params, w.dt
        b = region_breaks(w)
        self.breaks = b
        self.mcH = Mesh2D(b["xs_H"], b["c"]["ys_H"])
        self.mch = Mesh2D(b["xs_h"], b["c"]["ys_h"])
        self.mpH = Mesh2D(b["xs_H"], b["p"]["ys_H"])
        self.mph = Mesh2D(b["xs_h"], b["p"]["ys_h"])
        self.mms = MMS(w.mms, self.prm)
        r = w.fine_per_coarse_x
        fx = [i * r for i in range(w.nx_coarse + 1)]
        fy_c = np.concatenate([[0], np.cumsum(b["c"]["rows"])]).tolist()
        fy_p = np.concatenate([[0], np.cumsum(b["p"]["rows"])]).tolist()
        self.subs_c = make_subdomains(self.mch, "c", w, fx, fy_c)
        self.subs_p = make_subdomains(self.mph, "p", w, fx, fy_p)
        self.Pc2 = prolongation(self.mcH, self.mch, "p2")
        self.Pc1 = prolongation(self.mcH, self.mch, "p1")
        self.Pp2 = prolongation(self.mpH, self.mph, "p2")
        # coarse operators
        self.RcH = region_whole(self.mcH, "c")
        self.RpH = region_whole(self.mpH, "p")
        self.OcH = Ops(self.RcH, self.prm, self.dt)
        self.OpH = Ops(self.RpH, self.prm, self.dt)
        # fine subdomain operators
        self.sub_c = [(s, Ops(region_sub(self.mch, s), self.prm, self.dt)) for s in self.subs_c]
        self.sub_p = [(s, Ops(region_sub(self.mph, s), self.prm, self.dt)) for s in self.subs_p]
        # coarse Dirichlet nodes (region boundary without Gamma)
        self.dir_cH = self._region_dirichlet(self.mcH, "c")
        self.dir_pH = self._region_dirichlet(self.mpH, "p")
        # Gamma node maps: porous Gamma node with the same x as a fluid Gamma node
        self.gam_c_h = self.mch.half[0, :]
        self.gam_p_h = self.mph.half[2 * self.mph.ny, :]
        self.gam_c_H = self.mcH.half[0, :]
        self.gam_p_H = self.mpH.half[2 * self.mpH.ny, :]
        # coarse Darcy matrices (time invariant) and factors
        self.AdH = [self.OpH.darcy_matrix(i) for i in range(3)]
        self.MpH = self.OpH.mass_matrix()
        free = np.setdiff1d(np.arange(self.mpH.nn), self.dir_pH)
        self.free_pH = free
        self.luH = [spla.splu(sps.csc_matrix(A[free][:, free])) for A in self.AdH]
        # PoU glue weights
        self.wc = self._pou(self.subs_c, self.mch.nn)
        self.wp = self._pou(self.subs_p, self.mph.nn)
        self.newton_iters = []
        self.init_state()

    @staticmethod
    def _region_dirichlet(m, region):
        J, I = np.meshgrid(np.arange(2 * m.ny + 1), np.arange(2 * m.nx + 1), indexing="ij")
        if region == "c":
            on = (I == 0) | (I == 2 * m.nx) | (J == 2 * m.ny)
        else:
            on = (I == 0) | (I == 2 * m.nx) | (J == 0)
        return np.unique(m.half[on])

    @staticmethod
    def _pou(subs, nn):
        cnt = np.zeros(nn)
        for s in subs:
            np.add.at(cnt, s.gnode[s.inD], 1.0)
        assert (cnt > 0).all()
        return 1.0 / cnt

    # ------------------------------------------------------------------ initial data
    def init_state(self):
        """u_H^0 = I_H u_0 (nodal interpolation; the paper's elliptic projection is replaced
        by interpolation), e_j^0 = (I_h u_0 - I_h I_H u_0) on Omega_j, zero on the artificial
        boundary."""
        m, t = self.mms, 0.0
        self.n = 0
        self.uH = m.u(self.mcH.node[:, 0], self.mcH.node[:, 1], t)
        self.pH = m.p(self.mcH.vert[:, 0], self.mcH.vert[:, 1], t)
        self.pdH = np.stack([m.pd(i, self.mpH.node[:, 0], self.mpH.node[:, 1], t) for i in range(3)])
        uh = m.u(self.mch.node[:, 0], self.mch.node[:, 1], t)
        pdh = np.stack([m.pd(i, self.mph.node[:, 0], self.mph.node[:, 1], t) for i in range(3)])
        uHh = np.stack([self.Pc2 @ self.uH[:, a] for a in range(2)], axis=1)
        pdHh = np.stack([self.Pp2 @ self.pdH[i] for i in range(3)])
        self.ec, self.dc = [], []
        for s, _ in self.sub_c:
            e = (uh - uHh)[s.gnode]
            e[s.kind == 2] = 0.0
            self.ec.append(e)
            self.dc.append(np.zeros(len(s.vloc)))
        self.ep = []
        for s, _ in self.sub_p:
            e = (pdh - pdHh)[:, s.gnode]
            e[:, s.kind == 2] = 0.0
            self.ep.append(e)
        self.glue()

    # ------------------------------------------------------------------ Step 1
    def coarse_darcy(self, t):
        O, R, m, p, dt = self.OpH, self.RpH, self.mms, self.prm, self.dt
        kF, kf, km = p.k
        cFf = p.sigma_star * kf / p.mu
        cfm = p.sigma * km / p.mu
        pn = self.pdH
        uc_gamma = np.zeros(self.mpH.nn)
        # u_cH^n . n_c on Gamma (n_c = (0,-1)) carried to the porous Gamma nodes
        uc_gamma[self.gam_p_H] = -self.uH[self.gam_c_H, 1]
        new = np.zeros_like(pn)
        for i in range(3):
            qq = m.q(i, R.xq[..., 0], R.xq[..., 1], t)
            rhs = O.darcy_load(qq) + (p.phiC[i] / dt) * (self.MpH @ pn[i])
            if i == 0:
                rhs += cFf * (self.MpH @ pn[1])
                rhs += O.gamma_vec(R.gamma_load(R.gamma_trace_qp(uc_gamma)))
            elif i == 1:
                rhs += cfm * (self.MpH @ pn[2]) + cFf * (self.MpH @ pn[0])
            else:
                rhs += cfm * (self.MpH @ pn[1])
            rhs -= O.gamma_vec(R.gamma_load(m.gd(i, R.exq, t)))
            x = np.zeros(self.mpH.nn)
            d = self.dir_pH
            x[d] = m.pd(i, self.mpH.node[d, 0], self.mpH.node[d, 1], t)
            A = self.AdH[i]
            f = self.free_pH
            b = rhs[f] - A[f][:, d] @ x[d]
            x[f] = self.luH[i].solve(b)
            new[i] = x
        return new

    def coarse_ns(self, t):
        O, m = self.OcH, self.mms
        nn = self.mcH.nn
        d = self.dir_cH
        u = self.uH.copy()
        u[d] = m.u(self.mcH.node[d, 0], self.mcH.node[d, 1], t)
        p = self.pH.copy()
        pF_gamma = np.zeros(nn)
        pF_gamma[self.gam_c_H] = self.pdH[0][self.gam_p_H]          # p_FH^n (lagged)
        fixed = np.concatenate([2 * d, 2 * d + 1])
        free = np.setdiff1d(np.arange(O.ntot), fixed)
        x = np.concatenate([u.ravel(), p])
        it = 0
        for it in range(1, 31):
            r = O.ns_residual(x[:2 * nn].reshape(nn, 2), self.uH, x[2 * nn:], t, m, pF_gamma)
            A = O.oseen_matrix(x[:2 * nn].reshape(nn, 2))
            dx = solve_sparse(A[free][:, free], -r[free])
            x[free] += dx
            if np.linalg.norm(dx) <= 1e-14 * max(np.linalg.norm(x), 1e-300):
                break
        self.newton_iters.append(it)
        return x[:2 * nn].reshape(nn, 2).copy(), x[2 * nn:].copy()

    # ------------------------------------------------------------------ Step 3
    def local_fluid_system(self, j, t, uH1h, uH0h, pH1h, pFn_h_gamma):
        """Reduced system (A_ff, b, free, xfull) of the conduit correction on Omega_j
        (eq. uclocalFully): Dirichlet values of the correction are in xfull[fixed] and
        have been moved to the right-hand side."""
        s, O = self.sub_c[j]
        m, prm = self.mms, self.prm
        g = s.gnode
        w1 = uH1h[g]
        w0 = uH0h[g]
        p1 = pH1h[s.gvert]
        pFg = pFn_h_gamma[g]
        # RHS: fine residual of the coarse solution, lagged correction, data
        r = -O.ns_residual(w1, w0, p1, t, m, pFg)
        r += (prm.eta / self.dt) * O.mass_vec(self.ec[j])
        A = O.oseen_matrix(w1)
        # boundary values of the correction
        eB = np.zeros((len(g), 2))
        gl = s.kind == 1
        xy = O.R.xy
        eB[gl] = m.u(xy[gl, 0], xy[gl, 1], t) - w1[gl]
        fixed_nodes = np.nonzero(s.kind > 0)[0]
        # the pressure correction lives in Q_0^h(Omega_j): zero on the artificial boundary
        fixed_p = 2 * len(g) + np.nonzero(s.art[s.vloc])[0]
        fixed = np.concatenate([2 * fixed_nodes, 2 * fixed_nodes + 1, fixed_p])
        free = np.setdiff1d(np.arange(O.ntot), fixed)
        xfull = np.zeros(O.ntot)
        xfull[:2 * len(g)] = eB.ravel()
        b = r[free] - A[free][:, fixed] @ xfull[fixed]
        return A[free][:, free], b, free, xfull

    def local_fluid(self, j, t, uH1h, uH0h, pH1h, pFn_h_gamma):
        s, O = self.sub_c[j]
        Aff, b, free, xfull = self.local_fluid_system(j, t, uH1h, uH0h, pH1h, pFn_h_gamma)
        xfull[free] = solve_sparse(Aff, b)
        nn = len(s.gnode)
        return xfull[:2 * nn].reshape(-1, 2), xfull[2 * nn:]

    def local_porous_system(self, j, i, t, pH1h, pH0h, ucn_h_gamma_n):
        """Reduced system (A_ff, b, free, x) of pressure i (0 = F, 1 = f, 2 = m) on Omega_j
        (eqs. pFlocalFully, pflocalFully, pmlocalFully)."""
        s, O = self.sub_p[j]
        m, prm, dt = self.mms, self.prm, self.dt
        g = s.gnode
        R = O.R
        kF, kf, km = prm.k
        cFf = prm.sigma_star * kf / prm.mu
        cfm = prm.sigma * km / prm.mu
        Mloc = O.mass_matrix()
        en = self.ep[j]
        P1 = pH1h[:, g]
        P0 = pH0h[:, g]
        partners = {0: [(cFf, 1)], 1: [(cfm, 2), (cFf, 0)], 2: [(cfm, 1)]}
        fixed = np.nonzero(s.kind > 0)[0]
        free = np.nonzero(s.kind == 0)[0]
        A = O.darcy_matrix(i)
        qq = m.q(i, R.xq[..., 0], R.xq[..., 1], t)
        r = O.darcy_load(qq) - A @ P1[i] + (prm.phiC[i] / dt) * (Mloc @ (P0[i] + en[i]))
        for c, k in partners[i]:
            r += c * (Mloc @ (P0[k] + en[k]))
        if i == 0 and len(R.edge_nodes):
            r += O.gamma_vec(R.gamma_load(R.gamma_trace_qp(ucn_h_gamma_n[g])))
        if len(R.edge_nodes):
            r -= O.gamma_vec(R.gamma_load(m.gd(i, R.exq, t)))
        x = np.zeros(len(g))
        gl = s.kind == 1
        x[gl] = m.pd(i, R.xy[gl, 0], R.xy[gl, 1], t) - P1[i][gl]
        b = r[free] - A[free][:, fixed] @ x[fixed]
        return A[free][:, free], b, free, x

    def local_porous(self, j, t, pH1h, pH0h, ucn_h_gamma_n):
        s, _ = self.sub_p[j]
        out = np.zeros((3, len(s.gnode)))
        for i in range(3):
            Aff, b, free, x = self.local_porous_system(j, i, t, pH1h, pH0h, ucn_h_gamma_n)
            x[free] = solve_sparse(Aff, b)
            out[i] = x
        return out

    def step_inputs(self):
        """Coarse step plus the fine-mesh inputs of the local problems of the next step
        (used to inspect the local systems); does not advance the state."""
        uH0, pdH0 = self.uH, self.pdH
        t, u1, p1, pd1 = self.coarse_step()
        uH1h = np.stack([self.Pc2 @ u1[:, a] for a in range(2)], axis=1)
        uH0h = np.stack([self.Pc2 @ uH0[:, a] for a in range(2)], axis=1)
        pH1h = self.Pc1 @ p1
        pdH1h = np.stack([self.Pp2 @ pd1[i] for i in range(3)])
        pdH0h = np.stack([self.Pp2 @ pdH0[i] for i in range(3)])
        pFn_c = np.zeros(self.mch.nn)
        pFn_c[self.gam_c_h] = pdH0h[0][self.gam_p_h]
        ucn_p = np.zeros(self.mph.nn)
        ucn_p[self.gam_p_h] = -uH0h[self.gam_c_h, 1]
        return dict(t=t, u1=u1, p1=p1, pd1=pd1, uH1h=uH1h, uH0h=uH0h, pH1h=pH1h, pdH1h=pdH1h,
                    pdH0h=pdH0h, pFn_c=pFn_c, ucn_p=ucn_p)

    # ------------------------------------------------------------------ Step 4
    def glue(self):
        uHh = np.stack([self.Pc2 @ self.uH[:, a] for a in range(2)], axis=1)
        pHh = self.Pc1 @ self.pH
        pdHh = np.stack([self.Pp2 @ self.pdH[i] for i in range(3)])
        u = uHh.copy()
        for (s, _), e in zip(self.sub_c, self.ec):
            idx = s.inD
            np.add.at(u, s.gnode[idx], self.wc[s.gnode[idx]][:, None] * e[idx])
        p = pHh.copy()
        for (s, _), dl in zip(self.sub_c, self.dc):
            idx = s.inD[s.vloc]
            gv = s.gvert[idx]
            np.add.at(p, gv, self.wc[gv] * dl[idx])
        pd = pdHh.copy()
        for (s, _), e in zip(self.sub_p, self.ep):
            idx = s.inD
            for i in range(3):
                np.add.at(pd[i], s.gnode[idx], self.wp[s.gnode[idx]] * e[i][idx])
        self.fine = {"ux": u[:, 0], "uy": u[:, 1], "p": p, "pF": pd[0], "pf": pd[1], "pm": pd[2]}
        return self.fine

    # ------------------------------------------------------------------ one step
    def coarse_step(self):
        t = (self.n + 1) * self.dt
        pd_new = self.coarse_darcy(t)
        u_new, p_new = self.coarse_ns(t)
        return t, u_new, p_new, pd_new

    def step(self):
        d = self.step_inputs()
        t = d["t"]
        new_ec, new_dc, new_ep = [], [], []
        for j in range(len(self.sub_c)):
            e, dl = self.local_fluid(j, t, d["uH1h"], d["uH0h"], d["pH1h"], d["pFn_c"])
            new_ec.append(e)
            new_dc.append(dl)
        for j in range(len(self.sub_p)):
            new_ep.append(self.local_porous(j, t, d["pdH1h"], d["pdH0h"], d["ucn_p"]))
        self.uH, self.pH, self.pdH = d["u1"], d["p1"], d["pd1"]
        self.ec, self.dc, self.ep = new_ec, new_dc, new_ep
        self.n += 1
        return self.glue()

    def run(self, nsteps=None):
        for _ in range(self.w.nsteps if nsteps is None else nsteps):
            self.step()
        return self.fine

    # ------------------------------------------------------------------ errors
    def exact_fine(self, t=None):
        t = self.n * self.dt if t is None else t
        m = self.mms
        u = m.u(self.mch.node[:, 0], self.mch.node[:, 1], t)
        return {"ux": u[:, 0], "uy": u[:, 1],
                "p": m.p(self.mch.vert[:, 0], self.mch.vert[:, 1], t),
                "pF": m.pd(0, self.mph.node[:, 0], self.mph.node[:, 1], t),
                "pf": m.pd(1, self.mph.node[:, 0], self.mph.node[:, 1], t),
                "pm": m.pd(2, self.mph.node[:, 0], self.mph.node[:, 1], t)}

    def errors(self):
        """FE errors of the glued fine fields at t_n: velocity H1 seminorm, pressure and
        Darcy L2 norms and Darcy H1 seminorms (quadrature on every fine triangle)."""
        t = self.n * self.dt
        m = self.mms
        out = {}
        for mesh, keys in ((self.mch, ("u",)), (self.mph, ("pF", "pf", "pm"))):
            X = mesh.tri_coords()
            det, Jinv, xq, W = fe.geometry(X)
            G = fe.grads(Jinv, fe.DPHI)
            if keys == ("u",):
                uh = np.stack([self.fine["ux"], self.fine["uy"]], axis=1)[mesh.tri6]
                gh = fe.grad_at_qp(G, uh)
                ge = m.grad_u(xq[..., 0], xq[..., 1], t)
                out["u_H1"] = np.sqrt(np.sum(W[..., None, None] * (gh - ge) ** 2))
                ue = m.u(xq[..., 0], xq[..., 1], t)
                out["u_L2"] = np.sqrt(np.sum(W[..., None] * (fe.at_qp(uh) - ue) ** 2))
                ph = np.einsum("qk,ek->eq", fe.PSI, self.fine["p"][mesh.tri])
                out["p_L2"] = np.sqrt(np.sum(W * (ph - m.p(xq[..., 0], xq[..., 1], t)) ** 2))
            else:
                for i, k in enumerate(keys):
                    ph = self.fine[k][mesh.tri6]
                    val = fe.at_qp(ph) - m.pd(i, xq[..., 0], xq[..., 1], t)
                    out[k + "_L2"] = np.sqrt(np.sum(W * val ** 2))
                    gd = fe.grad_at_qp(G, ph) - m.grad_pd(i, xq[..., 0], xq[..., 1], t)
                    out[k + "_H1"] = np.sqrt(np.sum(W[..., None] * gd ** 2))
        return out
