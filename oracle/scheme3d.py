"""Algorithm 3 of the paper (Sec. 5) on the 3D configurations, written out plainly in FP64
with NumPy/SciPy: the same steps, readings and solver as the 2D oracle (``scheme``), on
Kuhn tetrahedral meshes with P2/P1 (fluid) and P2 (three pressures) elements.

Test infrastructure (see the package docstring).

Per time step n -> n+1 (t = (n+1) dt):
  Step 1: three decoupled coarse P2 Darcy solves (partners and the conduit velocity on Gamma
          lagged at t_n); the nonlinear coarse conduit problem with p_FH^n on Gamma by
          Newton's method (||delta||/||x|| <= 1e-14 or 30 iterations).
  Step 2: overlapping subdomains (``mesh3d.make_subdomains3d``).
  Step 3: on every Omega_j the fine correction whose right-hand side is the fine residual of
          the coarse solution plus the lagged local corrections e_j^n.
  Step 4: correction of data on D_j; shared closure nodes averaged (1 / #{j: x in closure D_j}).
Gamma is z = 1: n_c = (0,0,-1), n_p = (0,0,1), tangential projection P_tau v = (v_x, v_y, 0),
so the Beavers-Joseph-Saffman term acts on the x and y velocity components and the normal
traction on the z component.  Linear solves use SciPy's SuperLU.
"""
import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from . import fe3d as fe
from .mesh3d import Mesh3D, make_subdomains3d, region_breaks3d
from .mms3d import MMS3D

FIELDS = ("ux", "uy", "uz", "p", "pF", "pf", "pm")


def prolongation3d(mH, mh, kind):
    """Sparse matrix of the fine nodal interpolant of coarse P2 ('p2') or P1 ('p1')
    functions on nested Kuhn meshes: row = fine node (P2 node or vertex), column = coarse
    node.  Each fine point is located in its coarse cell and in the first of the cell's six
    tetrahedra (in mesh order) whose barycentric coordinates are all >= -1e-12."""
    pts = mh.node if kind == "p2" else mh.vert
    nb = 10 if kind == "p2" else 4
    ci = np.clip(np.searchsorted(mH.xs, pts[:, 0], side="right") - 1, 0, mH.nx - 1)
    cj = np.clip(np.searchsorted(mH.ys, pts[:, 1], side="right") - 1, 0, mH.ny - 1)
    ck = np.clip(np.searchsorted(mH.zs, pts[:, 2], side="right") - 1, 0, mH.nz - 1)
    cell = ci + mH.nx * (cj + mH.ny * ck)
    rows, cols, vals = [], [], []
    taken = np.zeros(len(pts), dtype=bool)
    for t in range(6):
        tet = 6 * cell + t
        X = mH.vert[mH.tet[tet]]
        det, Jinv, _, _ = fe.geometry(X)
        xi = np.einsum("erc,ec->er", Jinv, pts - X[:, 0, :])
        lam = np.concatenate([1 - xi.sum(axis=1, keepdims=True), xi], axis=1)
        inside = (lam.min(axis=1) >= -1e-12) & ~taken
        taken |= inside
        idx = np.nonzero(inside)[0]
        if kind == "p2":
            N, _ = fe.p2_basis(xi[idx])
            nodes = mH.tet10[tet[idx]]
        else:
            N, _ = fe.p1_basis(xi[idx])
            nodes = mH.tet[tet[idx]]
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


class Region3D:
    """Geometry, element data and Gamma faces of one region mesh (or of one subdomain)."""

    def __init__(self, mesh, tets, tet10, tet4, nn, nv, gamma_faces, gnode):
        self.mesh = mesh
        X = mesh.vert[mesh.tet[tets]]
        self.det, self.Jinv, self.xq, self.W = fe.geometry(X)
        self.G = fe.grads(self.Jinv, fe.DPHI)
        self.tet10, self.tet4, self.nn, self.nv = tet10, tet4, nn, nv
        self.gnode = gnode
        self.xyz = mesh.node[gnode]
        self.faces = gamma_faces
        if len(gamma_faces):
            P = self.xyz[gamma_faces[:, :3], :2]
            self.fW, self.fxq, self.fJinv = fe.face_geometry(P)
        else:
            self.fW = np.zeros((0, 7))

    def gamma_mass(self):
        return np.einsum("fq,qa,qb->fab", self.fW, fe.FPHI, fe.FPHI)

    def gamma_load(self, gq):
        """int_Gamma g phi_a for g given at face quadrature points (nf, 7)."""
        return np.einsum("fq,fq,qa->fa", self.fW, gq, fe.FPHI)

    def gamma_trace_qp(self, nodal):
        return np.einsum("qa,fa->fq", fe.FPHI, nodal[self.faces])

    def gamma_grad_qp(self, nodal):
        """Tangential gradient (d/dx, d/dy) at face quadrature points (nf, 7, 2)."""
        g = np.einsum("qar,frc->fqac", fe.FDPHI, self.fJinv)
        return np.einsum("fqac,fa->fqc", g, nodal[self.faces])


def region_whole(mesh, region):
    K = 0 if region == "c" else mesh.nz
    faces = mesh.face_triangles(K)
    return Region3D(mesh, np.arange(len(mesh.tet)), mesh.tet10, mesh.tet, mesh.nn, mesh.nv, faces,
                    np.arange(mesh.nn))


def region_sub(mesh, sub):
    return Region3D(mesh, sub.tets, sub.tet10, sub.tet4, len(sub.gnode), len(sub.vloc), sub.gamma_faces, sub.gnode)


class Ops3D:
    """Element-level operators of Sec. 3.1 on a 3D Region, with the scheme's coefficients."""

    def __init__(self, R, prm, dt):
        self.R, self.prm, self.dt = R, prm, dt
        self.M = fe.mass_p2(R.W)
        self.K = fe.stiff_p2(R.W, R.G)
        nn, nv = R.nn, R.nv
        self.vdof = 3 * R.tet10[:, :, None] + np.arange(3)[None, None, :]     # (ne,10,3)
        self.pdof = 3 * nn + R.tet4                                           # (ne,4)
        self.nvel = 3 * nn
        self.ntot = 3 * nn + nv

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
        d = self.R.tet10
        return coo_assemble(d[:, :, None], d[:, None, :], a * self.M + b * self.K, self.R.nn)

    def mass_matrix(self):
        d = self.R.tet10
        return coo_assemble(d[:, :, None], d[:, None, :], self.M, self.R.nn)

    def darcy_load(self, q_at_qp):
        return vec_assemble(self.R.tet10, fe.load_p2(self.R.W, q_at_qp), self.R.nn)

    def gamma_vec(self, face_vals):
        return vec_assemble(self.R.faces, face_vals, self.R.nn)

    def oseen_matrix(self, w_nodal):
        """Jacobian of the conduit residual about velocity w (nodal (nn,3)), with BJS."""
        R, prm = self.R, self.prm
        we = w_nodal[R.tet10]
        Kvv, Kvp, Kpv = fe.oseen_blocks(R.W, R.G, fe.at_qp(we), fe.grad_at_qp(R.G, we), self.dt, prm)
        n = self.ntot
        A = coo_assemble(self.vdof[:, :, :, None, None], self.vdof[:, None, None, :, :], Kvv, n)
        A = A + coo_assemble(self.vdof[:, :, :, None], self.pdof[:, None, None, :], Kvp, n)
        A = A + coo_assemble(self.pdof[:, :, None, None], self.vdof[:, None, :, :], Kpv, n)
        if len(R.faces):
            bjs = prm.eta * prm.nu * prm.alpha / np.sqrt(prm.k[0])
            Mf = R.gamma_mass() * bjs
            for a in range(2):                                       # P_tau: x and y components
                d = 3 * R.faces + a
                A = A + coo_assemble(d[:, :, None], d[:, None, :], Mf, n)
        return A.tocsr()

    def ns_residual(self, u, un, p, t, mms, pF_gamma):
        """Conduit residual (eq. uclocalFully's bracket / eq. pcFully) in 3D:
           eta/dt(u-un,v) + a_c(u,v) + b(v,p) - b(u,q) + b_N(u,u,v)
           + eta/rho <pF, v.n_c> + eta nu alpha sqrt(kF)/mu <grad_tau pF, P_tau v>
           + BJS <P_tau u, P_tau v> - eta (f, v) + eta <g_N, v.n_c> + eta <g_T, P_tau v>."""
        R, prm = self.R, self.prm
        ue, une = u[R.tet10], un[R.tet10]
        Gu = fe.grad_at_qp(R.G, ue)
        pq = np.einsum("qk,ek->eq", fe.PSI, p[R.tet4])
        fq = mms.f(R.xq[..., 0], R.xq[..., 1], R.xq[..., 2], t)
        Rv, Rp = fe.ns_residual_volume(R.W, R.G, fe.at_qp(ue), fe.at_qp(une), Gu, pq, fq, self.dt, prm)
        r = np.zeros(self.ntot)
        np.add.at(r, self.vdof.ravel(), Rv.ravel())
        np.add.at(r, self.pdof.ravel(), Rp.ravel())
        if len(R.faces):
            eta, nu, al, kF, mu, rho = prm.eta, prm.nu, prm.alpha, prm.k[0], prm.mu, prm.rho
            bjs = eta * nu * al / np.sqrt(kF)
            Mf = R.gamma_mass()
            pFq = R.gamma_trace_qp(pF_gamma)
            dpF = R.gamma_grad_qp(pF_gamma)
            xq = R.fxq
            gN = mms.gN(xq[..., 0], xq[..., 1], t)
            gT = mms.gT(xq[..., 0], xq[..., 1], t)
            for a in range(2):
                ra = bjs * np.einsum("fab,fb->fa", Mf, u[R.faces, a])
                ra += (eta * nu * al * np.sqrt(kF) / mu) * R.gamma_load(dpF[..., a]) + eta * R.gamma_load(gT[..., a])
                np.add.at(r, (3 * R.faces + a).ravel(), ra.ravel())
            # v.n_c = -v_z on Gamma
            rz = -(eta / rho) * R.gamma_load(pFq) - eta * R.gamma_load(gN)
            np.add.at(r, (3 * R.faces + 2).ravel(), rz.ravel())
        return r

    def mass_vec(self, nodal_vec):
        R = self.R
        vals = np.einsum("eij,eja->eia", self.M, nodal_vec[R.tet10])
        r = np.zeros(self.ntot)
        np.add.at(r, self.vdof.ravel(), vals.ravel())
        return r


def solve_sparse(A, b):
    return spla.splu(sps.csc_matrix(A)).solve(b)


class TwoGridOracle3D:
    """Algorithm 3 on a 3D workload (``workloads.Workload3D``)."""

    def __init__(self, w):
        self.w, self.prm, self.dt = w, w.params, w.dt
        b = region_breaks3d(w)
        xs_H, xs_h = b["xs_H"], b["xs_h"]
        self.mcH = Mesh3D(xs_H, xs_H, b["c"]["zs_H"])
        self.mch = Mesh3D(xs_h, xs_h, b["c"]["zs_h"])
        self.mpH = Mesh3D(xs_H, xs_H, b["p"]["zs_H"])
        self.mph = Mesh3D(xs_h, xs_h, b["p"]["zs_h"])
        self.mms = MMS3D(w.mms, self.prm)
        self.subs_c = make_subdomains3d(self.mch, "c", w)
        self.subs_p = make_subdomains3d(self.mph, "p", w)
        self.Pc2 = prolongation3d(self.mcH, self.mch, "p2")
        self.Pc1 = prolongation3d(self.mcH, self.mch, "p1")
        self.Pp2 = prolongation3d(self.mpH, self.mph, "p2")
        self.RcH = region_whole(self.mcH, "c")
        self.RpH = region_whole(self.mpH, "p")
        self.OcH = Ops3D(self.RcH, self.prm, self.dt)
        self.OpH = Ops3D(self.RpH, self.prm, self.dt)
        self.sub_c = [(s, Ops3D(region_sub(self.mch, s), self.prm, self.dt)) for s in self.subs_c]
        self.sub_p = [(s, Ops3D(region_sub(self.mph, s), self.prm, self.dt)) for s in self.subs_p]
        self.dir_cH = self._region_dirichlet(self.mcH, "c")
        self.dir_pH = self._region_dirichlet(self.mpH, "p")
        # Gamma node maps: porous Gamma node with the same (x, y) as a fluid Gamma node
        self.gam_c_h = self.mch.half[0].ravel()
        self.gam_p_h = self.mph.half[2 * self.mph.nz].ravel()
        self.gam_c_H = self.mcH.half[0].ravel()
        self.gam_p_H = self.mpH.half[2 * self.mpH.nz].ravel()
        self.AdH = [self.OpH.darcy_matrix(i) for i in range(3)]
        self.MpH = self.OpH.mass_matrix()
        free = np.setdiff1d(np.arange(self.mpH.nn), self.dir_pH)
        self.free_pH = free
        self.luH = [spla.splu(sps.csc_matrix(A[free][:, free])) for A in self.AdH]
        self.wc = self._pou(self.subs_c, self.mch.nn)
        self.wp = self._pou(self.subs_p, self.mph.nn)
        self.newton_iters = []
        self.init_state()

    @staticmethod
    def _region_dirichlet(m, region):
        h = m.hidx
        I, J, K = h[:, 0], h[:, 1], h[:, 2]
        on = (I == 0) | (I == 2 * m.nx) | (J == 0) | (J == 2 * m.ny)
        on |= (K == 2 * m.nz) if region == "c" else (K == 0)
        return np.nonzero(on)[0]

    @staticmethod
    def _pou(subs, nn):
        cnt = np.zeros(nn)
        for s in subs:
            np.add.at(cnt, s.gnode[s.inD], 1.0)
        assert (cnt > 0).all()
        return 1.0 / cnt

    def _u_at(self, mesh, t):
        n = mesh.node
        return self.mms.u(n[:, 0], n[:, 1], n[:, 2], t)

    def _pd_at(self, mesh, t):
        n = mesh.node
        return np.stack([self.mms.pd(i, n[:, 0], n[:, 1], n[:, 2], t) for i in range(3)])

    def init_state(self):
        """Nodal interpolation of the initial data (as in 2D); e_j^0 = (I_h u_0 - I_h I_H u_0)
        on Omega_j, zero on the artificial boundary."""
        t = 0.0
        self.n = 0
        self.uH = self._u_at(self.mcH, t)
        v = self.mcH.vert
        self.pH = self.mms.p(v[:, 0], v[:, 1], v[:, 2], t)
        self.pdH = self._pd_at(self.mpH, t)
        uh = self._u_at(self.mch, t)
        pdh = self._pd_at(self.mph, t)
        uHh = np.stack([self.Pc2 @ self.uH[:, a] for a in range(3)], axis=1)
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
        cFf = p.sigma_star * p.k[1] / p.mu
        cfm = p.sigma * p.k[2] / p.mu
        pn = self.pdH
        uc_gamma = np.zeros(self.mpH.nn)
        uc_gamma[self.gam_p_H] = -self.uH[self.gam_c_H, 2]          # u_cH^n . n_c, n_c = -e_z
        xq = R.xq
        fx = R.fxq
        new = np.zeros_like(pn)
        for i in range(3):
            qq = m.q(i, xq[..., 0], xq[..., 1], xq[..., 2], t)
            rhs = O.darcy_load(qq) + (p.phiC[i] / dt) * (self.MpH @ pn[i])
            if i == 0:
                rhs += cFf * (self.MpH @ pn[1])
                rhs += O.gamma_vec(R.gamma_load(R.gamma_trace_qp(uc_gamma)))
            elif i == 1:
                rhs += cfm * (self.MpH @ pn[2]) + cFf * (self.MpH @ pn[0])
            else:
                rhs += cfm * (self.MpH @ pn[1])
            rhs -= O.gamma_vec(R.gamma_load(m.gd(i, fx[..., 0], fx[..., 1], t)))
            x = np.zeros(self.mpH.nn)
            d = self.dir_pH
            nd = self.mpH.node[d]
            x[d] = m.pd(i, nd[:, 0], nd[:, 1], nd[:, 2], t)
            A = self.AdH[i]
            f = self.free_pH
            x[f] = self.luH[i].solve(rhs[f] - A[f][:, d] @ x[d])
            new[i] = x
        return new

    def coarse_ns(self, t):
        O, m = self.OcH, self.mms
        nn = self.mcH.nn
        d = self.dir_cH
        u = self.uH.copy()
        nd = self.mcH.node[d]
        u[d] = m.u(nd[:, 0], nd[:, 1], nd[:, 2], t)
        pF_gamma = np.zeros(nn)
        pF_gamma[self.gam_c_H] = self.pdH[0][self.gam_p_H]
        fixed = np.concatenate([3 * d, 3 * d + 1, 3 * d + 2])
        free = np.setdiff1d(np.arange(O.ntot), fixed)
        x = np.concatenate([u.ravel(), self.pH.copy()])
        it = 0
        for it in range(1, 31):
            r = O.ns_residual(x[:3 * nn].reshape(nn, 3), self.uH, x[3 * nn:], t, m, pF_gamma)
            A = O.oseen_matrix(x[:3 * nn].reshape(nn, 3))
            dx = solve_sparse(A[free][:, free], -r[free])
            x[free] += dx
            if np.linalg.norm(dx) <= 1e-14 * max(np.linalg.norm(x), 1e-300):
                break
        self.newton_iters.append(it)
        return x[:3 * nn].reshape(nn, 3).copy(), x[3 * nn:].copy()

    # ------------------------------------------------------------------ Step 3
    def local_fluid_system(self, j, t, uH1h, uH0h, pH1h, pFn_h_gamma):
        """Reduced system (A_ff, b, free, xfull) of the conduit correction on Omega_j
        (eq. uclocalFully); Dirichlet values of the correction are moved to the right."""
        s, O = self.sub_c[j]
        m, prm = self.mms, self.prm
        g = s.gnode
        w1 = uH1h[g]
        r = -O.ns_residual(w1, uH0h[g], pH1h[s.gvert], t, m, pFn_h_gamma[g])
        r += (prm.eta / self.dt) * O.mass_vec(self.ec[j])
        A = O.oseen_matrix(w1)
        eB = np.zeros((len(g), 3))
        gl = s.kind == 1
        xyz = O.R.xyz
        eB[gl] = m.u(xyz[gl, 0], xyz[gl, 1], xyz[gl, 2], t) - w1[gl]
        fixed_nodes = np.nonzero(s.kind > 0)[0]
        fixed_p = 3 * len(g) + np.nonzero(s.art[s.vloc])[0]
        fixed = np.concatenate([3 * fixed_nodes, 3 * fixed_nodes + 1, 3 * fixed_nodes + 2, fixed_p])
        free = np.setdiff1d(np.arange(O.ntot), fixed)
        xfull = np.zeros(O.ntot)
        xfull[:3 * len(g)] = eB.ravel()
        b = r[free] - A[free][:, fixed] @ xfull[fixed]
        return A[free][:, free], b, free, xfull

    def local_fluid(self, j, t, uH1h, uH0h, pH1h, pFn_h_gamma):
        s, _ = self.sub_c[j]
        Aff, b, free, xfull = self.local_fluid_system(j, t, uH1h, uH0h, pH1h, pFn_h_gamma)
        xfull[free] = solve_sparse(Aff, b)
        nn = len(s.gnode)
        return xfull[:3 * nn].reshape(-1, 3), xfull[3 * nn:]

    def local_porous_system(self, j, i, t, pH1h, pH0h, ucn_h_gamma_n):
        """Reduced system of pressure i (0 = F, 1 = f, 2 = m) on Omega_j (eqs. pFlocalFully,
        pflocalFully, pmlocalFully)."""
        s, O = self.sub_p[j]
        m, prm, dt = self.mms, self.prm, self.dt
        g = s.gnode
        R = O.R
        cFf = prm.sigma_star * prm.k[1] / prm.mu
        cfm = prm.sigma * prm.k[2] / prm.mu
        Mloc = O.mass_matrix()
        en = self.ep[j]
        P1 = pH1h[:, g]
        P0 = pH0h[:, g]
        partners = {0: [(cFf, 1)], 1: [(cfm, 2), (cFf, 0)], 2: [(cfm, 1)]}
        fixed = np.nonzero(s.kind > 0)[0]
        free = np.nonzero(s.kind == 0)[0]
        A = O.darcy_matrix(i)
        qq = m.q(i, R.xq[..., 0], R.xq[..., 1], R.xq[..., 2], t)
        r = O.darcy_load(qq) - A @ P1[i] + (prm.phiC[i] / dt) * (Mloc @ (P0[i] + en[i]))
        for c, k in partners[i]:
            r += c * (Mloc @ (P0[k] + en[k]))
        if len(R.faces):
            if i == 0:
                r += O.gamma_vec(R.gamma_load(R.gamma_trace_qp(ucn_h_gamma_n[g])))
            r -= O.gamma_vec(R.gamma_load(m.gd(i, R.fxq[..., 0], R.fxq[..., 1], t)))
        x = np.zeros(len(g))
        gl = s.kind == 1
        x[gl] = m.pd(i, R.xyz[gl, 0], R.xyz[gl, 1], R.xyz[gl, 2], t) - P1[i][gl]
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
        """Coarse step plus the fine-mesh inputs of the local problems (state not advanced)."""
        uH0, pdH0 = self.uH, self.pdH
        t, u1, p1, pd1 = self.coarse_step()
        uH1h = np.stack([self.Pc2 @ u1[:, a] for a in range(3)], axis=1)
        uH0h = np.stack([self.Pc2 @ uH0[:, a] for a in range(3)], axis=1)
        pH1h = self.Pc1 @ p1
        pdH1h = np.stack([self.Pp2 @ pd1[i] for i in range(3)])
        pdH0h = np.stack([self.Pp2 @ pdH0[i] for i in range(3)])
        pFn_c = np.zeros(self.mch.nn)
        pFn_c[self.gam_c_h] = pdH0h[0][self.gam_p_h]
        ucn_p = np.zeros(self.mph.nn)
        ucn_p[self.gam_p_h] = -uH0h[self.gam_c_h, 2]
        return dict(t=t, u1=u1, p1=p1, pd1=pd1, uH1h=uH1h, uH0h=uH0h, pH1h=pH1h, pdH1h=pdH1h,
                    pdH0h=pdH0h, pFn_c=pFn_c, ucn_p=ucn_p)

    # ------------------------------------------------------------------ Step 4
    def glue(self):
        uHh = np.stack([self.Pc2 @ self.uH[:, a] for a in range(3)], axis=1)
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
        self.fine = {"ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "p": p, "pF": pd[0], "pf": pd[1], "pm": pd[2]}
        return self.fine

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

    def exact_fine(self, t=None):
        t = self.n * self.dt if t is None else t
        u = self._u_at(self.mch, t)
        v = self.mch.vert
        pd = self._pd_at(self.mph, t)
        return {"ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "p": self.mms.p(v[:, 0], v[:, 1], v[:, 2], t),
                "pF": pd[0], "pf": pd[1], "pm": pd[2]}
