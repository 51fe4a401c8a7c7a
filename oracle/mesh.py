"""Structured right-triangle meshes of the two regions, P2/P1 numbering and the
overlapping subdomains of Algorithm 3, Step 2 (Sec. 5).

Numbering (fixed so that any two implementations agree bit for bit):
  * vertex (i, j) of a region with nx x ny cells has id  i + (nx + 1) * j;
  * every cell (i, j) is split by its diagonal (i, j)-(i+1, j+1); triangles are listed
    cell by cell (x fastest), lower triangle [v(i,j), v(i+1,j), v(i+1,j+1)] first, then
    upper [v(i,j), v(i+1,j+1), v(i,j+1)] (both counter-clockwise);
  * P2 nodes: the vertices, then one node per edge, edges sorted by (min vid, max vid);
  * P2 local node order in a triangle: v0, v1, v2, mid(v0v1), mid(v1v2), mid(v2v0).
Coordinates of grid lines are exact rationals k / n rounded once, so that nested coarse
and fine grid lines coincide bit for bit; edge nodes sit at 0.5 * (a + b).

All P2 nodes of such a mesh lie on the "half grid": node (I, J) with I in 0..2nx,
J in 0..2ny; even/even are vertices, the others are edge midpoints.
"""
import numpy as np


def region_breaks(w):
    """Grid lines of the coarse and fine meshes of both regions for a workload.

    Fluid region [0,1]x[1,2], porous region [0,1]x[0,1]; Gamma is y = 1.  Fine rows per
    coarse row are listed in w.fine_rows_from_gamma from Gamma outwards.
    Returns dict with xs_H, xs_h, and per region ('c' fluid, 'p' porous) ys_H, ys_h and
    the fine row index of every coarse row line."""
    nxc, nyc, r = w.nx_coarse, w.ny_coarse, w.fine_per_coarse_x
    xs_H = np.array([i / nxc for i in range(nxc + 1)])
    xs_h = np.array([k / (nxc * r) for k in range(nxc * r + 1)])
    rows = list(w.fine_rows_from_gamma)
    assert len(rows) == nyc
    out = {"xs_H": xs_H, "xs_h": xs_h}
    # fluid: coarse row c (from y=1 upwards) is at distance c from Gamma
    ys = [1.0]
    for c in range(nyc):
        m = rows[c]
        for k in range(1, m + 1):
            ys.append(1.0 + (c * m + k) / (nyc * m))
    out["c"] = {"ys_H": np.array([1.0 + c / nyc for c in range(nyc + 1)]), "ys_h": np.array(ys),
                "rows": [rows[c] for c in range(nyc)]}
    # porous: coarse row c (from y=0 upwards) is at distance nyc-1-c from Gamma
    ys = [0.0]
    prow = [rows[nyc - 1 - c] for c in range(nyc)]
    for c in range(nyc):
        m = prow[c]
        for k in range(1, m + 1):
            ys.append((c * m + k) / (nyc * m))
    out["p"] = {"ys_H": np.array([c / nyc for c in range(nyc + 1)]), "ys_h": np.array(ys),
                "rows": prow}
    return out


class Mesh2D:
    """Right-triangle mesh of a rectangle given its x and y grid lines."""

    def __init__(self, xs, ys):
        self.xs = np.asarray(xs, dtype=float)
        self.ys = np.asarray(ys, dtype=float)
        nx, ny = len(xs) - 1, len(ys) - 1
        self.nx, self.ny = nx, ny
        I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
        self.nv = (nx + 1) * (ny + 1)
        self.vert = np.stack([self.xs[I.ravel()], self.ys[J.ravel()]], axis=1)
        vid = lambda i, j: i + (nx + 1) * j
        tris = []
        for j in range(ny):
            for i in range(nx):
                tris.append([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)])
                tris.append([vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)])
        self.tri = np.array(tris, dtype=np.int64)
        e = np.concatenate([self.tri[:, [0, 1]], self.tri[:, [1, 2]], self.tri[:, [2, 0]]])
        e = np.sort(e, axis=1)
        self.edges = np.unique(e, axis=0)          # lexicographic (min, max)
        self.ne = len(self.edges)
        key = self.edges[:, 0] * self.nv + self.edges[:, 1]
        order = np.argsort(key)
        self._ekey, self._eord = key[order], order

        def eid(a, b):
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            pos = np.searchsorted(self._ekey, lo * self.nv + hi)
            return self.nv + self._eord[pos]
        t = self.tri
        self.tri6 = np.stack([t[:, 0], t[:, 1], t[:, 2], eid(t[:, 0], t[:, 1]),
                              eid(t[:, 1], t[:, 2]), eid(t[:, 2], t[:, 0])], axis=1)
        self.nn = self.nv + self.ne
        mid = 0.5 * (self.vert[self.edges[:, 0]] + self.vert[self.edges[:, 1]])
        self.node = np.concatenate([self.vert, mid])
        # half-grid map (I, J) -> P2 node id
        hg = -np.ones((2 * ny + 1, 2 * nx + 1), dtype=np.int64)
        Iv, Jv = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
        hg[2 * Jv, 2 * Iv] = vid(Iv, Jv)
        Ih, Jh = np.meshgrid(np.arange(nx), np.arange(ny + 1), indexing="xy")
        hg[2 * Jh, 2 * Ih + 1] = eid(vid(Ih, Jh).ravel(), vid(Ih + 1, Jh).ravel()).reshape(Ih.shape)
        Iu, Ju = np.meshgrid(np.arange(nx + 1), np.arange(ny), indexing="xy")
        hg[2 * Ju + 1, 2 * Iu] = eid(vid(Iu, Ju).ravel(), vid(Iu, Ju + 1).ravel()).reshape(Iu.shape)
        Id, Jd = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
        hg[2 * Jd + 1, 2 * Id + 1] = eid(vid(Id, Jd).ravel(), vid(Id + 1, Jd + 1).ravel()).reshape(Id.shape)
        assert (hg >= 0).all()
        self.half = hg                      # half[J, I]

    def tri_coords(self, tris=None):
        t = self.tri if tris is None else self.tri[tris]
        return self.vert[t]                 # (ne, 3, 2)

    def cells_tris(self, i0, i1, j0, j1):
        """Triangle indices of the cell box [i0,i1) x [j0,j1), in mesh order."""
        out = []
        for j in range(j0, j1):
            for i in range(i0, i1):
                c = i + self.nx * j
                out += [2 * c, 2 * c + 1]
        return np.array(out, dtype=np.int64)


class Subdomain:
    """One overlapping subdomain Omega_j (a box of fine cells) with its D_j box.

    region: 'c' (conduit/fluid) or 'p' (porous).  Boxes are in fine cell indices.
    node classification (P2 nodes of Omega_j, half-grid indices):
      kind 0 = unknown, 1 = global Dirichlet (data I_h g - I_h I_H g),
      kind 2 = artificial boundary (correction 0).
    Global Dirichlet wins over artificial, which wins over the natural condition on Gamma.
    """

    def __init__(self, mesh, region, box, dbox):
        self.region = region
        self.i0, self.i1, self.j0, self.j1 = box
        self.di0, self.di1, self.dj0, self.dj1 = dbox
        nx, ny = mesh.nx, mesh.ny
        Is = np.arange(2 * self.i0, 2 * self.i1 + 1)
        Js = np.arange(2 * self.j0, 2 * self.j1 + 1)
        I, J = np.meshgrid(Is, Js, indexing="xy")
        I, J = I.ravel(), J.ravel()                   # I fastest
        self.hI, self.hJ = I, J
        self.gnode = mesh.half[J, I]                  # local -> global P2 node
        gamma_J = 0 if region == "c" else 2 * ny
        if region == "c":
            on_region_bdry = (I == 0) | (I == 2 * nx) | (J == 2 * ny)
        else:
            on_region_bdry = (I == 0) | (I == 2 * nx) | (J == 0)
        # sides of the box that lie inside the region carry the artificial condition
        on_art_side = (((I == 2 * self.i0) & (self.i0 > 0)) | ((I == 2 * self.i1) & (self.i1 < nx)) |
                       ((J == 2 * self.j0) & (self.j0 > 0)) | ((J == 2 * self.j1) & (self.j1 < ny)))
        self.art = on_art_side          # closure of the artificial boundary (pressure: 0)
        kind = np.zeros(len(I), dtype=np.int64)
        kind[on_art_side] = 2
        kind[on_region_bdry] = 1
        self.kind = kind
        self.touches_gamma = (self.j0 == 0) if region == "c" else (self.j1 == ny)
        self.tris = mesh.cells_tris(self.i0, self.i1, self.j0, self.j1)
        # local P2 node index of each triangle node
        nI = 2 * (self.i1 - self.i0) + 1
        g2l = {int(g): k for k, g in enumerate(self.gnode)}
        self.tri6 = np.vectorize(g2l.__getitem__)(mesh.tri6[self.tris])
        # vertices of Omega_j (P1 nodes), local order = half-grid order of even/even nodes
        isv = (I % 2 == 0) & (J % 2 == 0)
        self.vloc = np.nonzero(isv)[0]                # local P2 index of each local vertex
        self.gvert = self.gnode[self.vloc]            # global vertex id (== global P2 id)
        v2l = {int(n): k for k, n in enumerate(self.vloc)}
        self.tri3 = np.vectorize(v2l.__getitem__)(self.tri6[:, :3])
        # partition-of-unity: node in the closure of D_j
        self.inD = ((I >= 2 * self.di0) & (I <= 2 * self.di1) &
                    (J >= 2 * self.dj0) & (J <= 2 * self.dj1))
        # Gamma edges of Omega_j: (left vertex, right vertex, midpoint) local node ids
        self.gamma_edges = np.zeros((0, 3), dtype=np.int64)
        if self.touches_gamma:
            row = np.nonzero(J == gamma_J)[0]
            row = row[np.argsort(I[row])]
            self.gamma_edges = np.stack([row[0:-1:2], row[2::2], row[1::2]], axis=1)


def make_subdomains(mesh, region, w, fine_x_of_coarse, fine_y_of_coarse):
    """Algorithm 3 Step 2: disjoint boxes D_j aligned with coarse lines, enlarged by
    w.overlap fine layers on sides interior to the region (clipped at its boundary)."""
    sx, sy = w.nsub
    nxc, nyc = w.nx_coarse, w.ny_coarse
    assert nxc % sx == 0 and nyc % sy == 0
    cx, cy = nxc // sx, nyc // sy
    subs = []
    for b in range(sy):
        for a in range(sx):
            di0, di1 = fine_x_of_coarse[a * cx], fine_x_of_coarse[(a + 1) * cx]
            dj0, dj1 = fine_y_of_coarse[b * cy], fine_y_of_coarse[(b + 1) * cy]
            i0 = max(di0 - w.overlap, 0) if di0 > 0 else 0
            i1 = min(di1 + w.overlap, mesh.nx) if di1 < mesh.nx else mesh.nx
            j0 = max(dj0 - w.overlap, 0) if dj0 > 0 else 0
            j1 = min(dj1 + w.overlap, mesh.ny) if dj1 < mesh.ny else mesh.ny
            subs.append(Subdomain(mesh, region, (i0, i1, j0, j1), (di0, di1, dj0, dj1)))
    return subs
