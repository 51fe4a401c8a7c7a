"""Structured Kuhn tetrahedral meshes of the two 3D regions, P2/P1 numbering and the
overlapping subdomains of Algorithm 3, Step 2 (Sec. 5) in three dimensions.

Test infrastructure: imported only by the tests, the oracle's own callers and the bench's
CPU baseline, never by the GPU library.

Numbering (fixed so that two implementations agree bit for bit):
  * vertex (i, j, k) of a box with nx x ny x nz cells has id  i + (nx+1) (j + (ny+1) k);
  * cells are listed x fastest, then y, then z; every cell is split into the six Kuhn
    tetrahedra along its diagonal v(0,0,0)-v(1,1,1): for each permutation (a, b, c) of the
    axes, in lexicographic order (0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0), the
    tetrahedron [v000, v000 + e_a, v000 + e_a + e_b, v111];
  * P2 nodes: the vertices, then one node per edge, edges sorted by (min vid, max vid);
  * P2 local node order in a tetrahedron: v0, v1, v2, v3, then the midpoints of the edges
    (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).
Every face of the Kuhn split of a cell is cut along its diagonal from the lower to the upper
corner, so neighbouring cells agree and every point of the half grid (I, J, K),
I in 0..2nx, ... is a P2 node: vertices have three even indices, axis-edge midpoints one odd,
face-diagonal midpoints two, the cell diagonal's midpoint three.
Coordinates of grid lines are k / n rounded once; edge nodes sit at 0.5 * (a + b).

Domains (3D configurations): porous region [0,1]^3, fluid region [0,1]^2 x [1,2];
Gamma is z = 1 with n_c = (0,0,-1), n_p = (0,0,1) and the tangential projection
P_tau v = (v_x, v_y, 0).
"""
import numpy as np

PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def region_breaks3d(w):
    """Grid lines of the coarse and fine meshes of both 3D regions (uniform in every axis)."""
    nc, r = w.n_coarse, w.fine_per_coarse
    xs_H = np.array([i / nc for i in range(nc + 1)])
    xs_h = np.array([k / (nc * r) for k in range(nc * r + 1)])
    return {"xs_H": xs_H, "xs_h": xs_h,
            "c": {"zs_H": 1.0 + xs_H, "zs_h": 1.0 + xs_h},
            "p": {"zs_H": xs_H.copy(), "zs_h": xs_h.copy()}}


class Mesh3D:
    """Kuhn tetrahedral mesh of a box given its x, y and z grid lines."""

    def __init__(self, xs, ys, zs):
        self.xs, self.ys, self.zs = (np.asarray(v, dtype=float) for v in (xs, ys, zs))
        nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nv = (nx + 1) * (ny + 1) * (nz + 1)
        I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
        I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))      # i fastest
        self.vert = np.stack([self.xs[I], self.ys[J], self.zs[K]], axis=1)
        vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
        tets = []
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    for p in PERMS:
                        c = [i, j, k]
                        t = [vid(*c)]
                        for ax in p:
                            c[ax] += 1
                            t.append(vid(*c))
                        tets.append(t)
        self.tet = np.array(tets, dtype=np.int64)
        e = np.concatenate([self.tet[:, list(ab)] for ab in EDGES])
        e = np.sort(e, axis=1)
        self.edges = np.unique(e, axis=0)
        self.ne = len(self.edges)
        key = self.edges[:, 0] * self.nv + self.edges[:, 1]
        order = np.argsort(key)
        ekey, eord = key[order], order

        def eid(a, b):
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            pos = np.searchsorted(ekey, lo * self.nv + hi)
            return self.nv + eord[pos]
        self._eid = eid
        t = self.tet
        self.tet10 = np.concatenate([t] + [eid(t[:, a], t[:, b])[:, None] for a, b in EDGES], axis=1)
        self.nn = self.nv + self.ne
        mid = 0.5 * (self.vert[self.edges[:, 0]] + self.vert[self.edges[:, 1]])
        self.node = np.concatenate([self.vert, mid])
        # half-grid map (I, J, K) -> P2 node id, from the vertex indices of every node
        hg = -np.ones((2 * nz + 1, 2 * ny + 1, 2 * nx + 1), dtype=np.int64)
        vi = np.stack([I, J, K], axis=1)
        hg[2 * K, 2 * J, 2 * I] = np.arange(self.nv)
        h = vi[self.edges[:, 0]] + vi[self.edges[:, 1]]
        hg[h[:, 2], h[:, 1], h[:, 0]] = self.nv + np.arange(self.ne)
        assert (hg >= 0).all()
        self.half = hg                      # half[K, J, I]
        self.hidx = np.zeros((self.nn, 3), dtype=np.int64)
        self.hidx[:self.nv] = 2 * vi
        self.hidx[self.nv:] = h

    def cells_tets(self, i0, i1, j0, j1, k0, k1):
        """Tetrahedron indices of the cell box [i0,i1) x [j0,j1) x [k0,k1), in mesh order."""
        out = []
        for k in range(k0, k1):
            for j in range(j0, j1):
                for i in range(i0, i1):
                    c = i + self.nx * (j + self.ny * k)
                    out += list(range(6 * c, 6 * c + 6))
        return np.array(out, dtype=np.int64)

    def face_triangles(self, K):
        """Triangles of the Kuhn split on the plane of vertex layer K (for Gamma): per cell of
        the layer (x fastest), the triangles [v(i,j), v(i+1,j), v(i+1,j+1)] and
        [v(i,j), v(i,j+1), v(i+1,j+1)] as P2 nodes (3 vertices, then the midpoints of the
        edges (0,1), (0,2), (1,2) of the triangle)."""
        nx, ny = self.nx, self.ny
        hv = lambda i, j: self.half[2 * K, 2 * j, 2 * i]
        hm = lambda I, J: self.half[2 * K, J, I]
        tris = []
        for j in range(ny):
            for i in range(nx):
                for (a, b, c) in (((i, j), (i + 1, j), (i + 1, j + 1)), ((i, j), (i, j + 1), (i + 1, j + 1))):
                    v = [hv(*a), hv(*b), hv(*c)]
                    m = [hm(a[0] + b[0], a[1] + b[1]), hm(a[0] + c[0], a[1] + c[1]), hm(b[0] + c[0], b[1] + c[1])]
                    tris.append(v + m)
        return np.array(tris, dtype=np.int64)


class Subdomain3D:
    """One overlapping subdomain Omega_j (a box of fine cells) with its D_j box, in 3D.

    region: 'c' (fluid, Gamma at its bottom z = 1) or 'p' (porous, Gamma at its top).
    Node kinds as in 2D: 0 unknown, 1 global Dirichlet (data I_h g - I_h I_H g),
    2 artificial boundary (correction 0); global Dirichlet wins over artificial, which wins
    over the natural condition on Gamma."""

    def __init__(self, mesh, region, box, dbox):
        self.region = region
        self.box, self.dbox = box, dbox
        i0, i1, j0, j1, k0, k1 = box
        nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
        I, J, K = np.meshgrid(np.arange(2 * i0, 2 * i1 + 1), np.arange(2 * j0, 2 * j1 + 1),
                              np.arange(2 * k0, 2 * k1 + 1), indexing="ij")
        I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))      # I fastest, then J, K
        self.hI, self.hJ, self.hK = I, J, K
        self.gnode = mesh.half[K, J, I]
        gamma_K = 0 if region == "c" else 2 * nz
        on_side = (I == 0) | (I == 2 * nx) | (J == 0) | (J == 2 * ny)
        on_region_bdry = on_side | ((K == 2 * nz) if region == "c" else (K == 0))
        on_art = (((I == 2 * i0) & (i0 > 0)) | ((I == 2 * i1) & (i1 < nx)) |
                  ((J == 2 * j0) & (j0 > 0)) | ((J == 2 * j1) & (j1 < ny)) |
                  ((K == 2 * k0) & (k0 > 0)) | ((K == 2 * k1) & (k1 < nz)))
        self.art = on_art
        kind = np.zeros(len(I), dtype=np.int64)
        kind[on_art] = 2
        kind[on_region_bdry] = 1
        self.kind = kind
        self.touches_gamma = (k0 == 0) if region == "c" else (k1 == nz)
        self.tets = mesh.cells_tets(i0, i1, j0, j1, k0, k1)
        g2l = {int(g): l for l, g in enumerate(self.gnode)}
        self.tet10 = np.vectorize(g2l.__getitem__)(mesh.tet10[self.tets])
        isv = (I % 2 == 0) & (J % 2 == 0) & (K % 2 == 0)
        self.vloc = np.nonzero(isv)[0]
        self.gvert = self.gnode[self.vloc]
        v2l = {int(n): k for k, n in enumerate(self.vloc)}
        self.tet4 = np.vectorize(v2l.__getitem__)(self.tet10[:, :4])
        di0, di1, dj0, dj1, dk0, dk1 = dbox
        self.inD = ((I >= 2 * di0) & (I <= 2 * di1) & (J >= 2 * dj0) & (J <= 2 * dj1) &
                    (K >= 2 * dk0) & (K <= 2 * dk1))
        # Gamma faces of Omega_j (local P2 node ids, see Mesh3D.face_triangles)
        self.gamma_faces = np.zeros((0, 6), dtype=np.int64)
        if self.touches_gamma:
            allf = mesh.face_triangles(gamma_K // 2)
            keep = []
            for j in range(j0, j1):
                for i in range(i0, i1):
                    c = i + nx * j
                    keep += [2 * c, 2 * c + 1]
            self.gamma_faces = np.vectorize(g2l.__getitem__)(allf[keep])


def make_subdomains3d(mesh, region, w):
    """Algorithm 3 Step 2: disjoint boxes D_j aligned with coarse lines, enlarged by
    w.overlap fine layers on sides interior to the region (clipped at its boundary)."""
    sx, sy, sz = w.nsub
    nc, r = w.n_coarse, w.fine_per_coarse
    assert nc % sx == 0 and nc % sy == 0 and nc % sz == 0
    n = nc * r
    subs = []
    for c in range(sz):
        for b in range(sy):
            for a in range(sx):
                lo = [a * n // sx, b * n // sy, c * n // sz]
                hi = [(a + 1) * n // sx, (b + 1) * n // sy, (c + 1) * n // sz]
                box = []
                for d in range(3):
                    box += [max(lo[d] - w.overlap, 0), min(hi[d] + w.overlap, n)]
                dbox = [lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]]
                subs.append(Subdomain3D(mesh, region, tuple(box), tuple(dbox)))
    return subs

