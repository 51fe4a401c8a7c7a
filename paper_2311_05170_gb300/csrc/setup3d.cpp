// Host-side layout of the 3D configurations: Kuhn tetrahedral meshes of the fluid box
// [0,1]^2 x [1,2] and the porous box [0,1]^3 on both levels, overlapping subdomains
// (Algorithm 3, Step 2) as boxes of fine cells, P2/P1 unknowns, CSR patterns and scatter maps,
// Gamma (z = 1) partner nodes, prolongation and glue tables, and the 3D reference tables.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "setup.hpp"

namespace tpns {

namespace {

constexpr int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
constexpr int TEDGES[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

}  // namespace

void Mesh::build3(const std::vector<double>& xs_, const std::vector<double>& ys_, const std::vector<double>& zs_) {
  dim = 3;
  vpe = 4;
  npe = 10;
  xs = xs_;
  ys = ys_;
  zs = zs_;
  nx = (int)xs.size() - 1;
  ny = (int)ys.size() - 1;
  nz = (int)zs.size() - 1;
  nv = (nx + 1) * (ny + 1) * (nz + 1);
  nt = 6 * nx * ny * nz;
  auto vid = [&](int i, int j, int k) { return i + (nx + 1) * (j + (ny + 1) * k); };
  tri.resize((size_t)nt * 4);
  size_t t = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int p = 0; p < 6; ++p) {
          int c[3] = {i, j, k};
          tri[4 * t] = vid(c[0], c[1], c[2]);
          for (int s = 0; s < 3; ++s) {
            c[PERMS[p][s]] += 1;
            tri[4 * t + 1 + s] = vid(c[0], c[1], c[2]);
          }
          ++t;
        }
  std::vector<std::pair<int32_t, int32_t>> edges;
  edges.reserve((size_t)nt * 6);
  for (size_t e = 0; e < (size_t)nt; ++e)
    for (auto& ab : TEDGES) {
      int32_t a = tri[4 * e + ab[0]], b = tri[4 * e + ab[1]];
      edges.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  nedge = (int)edges.size();
  nn = nv + nedge;
  auto eid = [&](int32_t a, int32_t b) {
    std::pair<int32_t, int32_t> key{std::min(a, b), std::max(a, b)};
    return nv + (int32_t)(std::lower_bound(edges.begin(), edges.end(), key) - edges.begin());
  };
  node.assign((size_t)nn * 3, 0.0);
  std::vector<int32_t> vI(nv), vJ(nv), vK(nv);
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const int v = vid(i, j, k);
        node[3 * (size_t)v] = xs[i];
        node[3 * (size_t)v + 1] = ys[j];
        node[3 * (size_t)v + 2] = zs[k];
        vI[v] = i; vJ[v] = j; vK[v] = k;
      }
  half.assign((size_t)(2 * nz + 1) * (2 * ny + 1) * (2 * nx + 1), -1);
  auto H = [&](int I, int J, int K) -> int32_t& { return half[((size_t)K * (2 * ny + 1) + J) * (2 * nx + 1) + I]; };
  for (int v = 0; v < nv; ++v) H(2 * vI[v], 2 * vJ[v], 2 * vK[v]) = v;
  for (int e = 0; e < nedge; ++e) {
    const int a = edges[e].first, b = edges[e].second;
    for (int c = 0; c < 3; ++c)
      node[3 * (size_t)(nv + e) + c] = 0.5 * (node[3 * (size_t)a + c] + node[3 * (size_t)b + c]);
    H(vI[a] + vI[b], vJ[a] + vJ[b], vK[a] + vK[b]) = nv + e;
  }
  tri6.resize((size_t)nt * 10);
  for (size_t e = 0; e < (size_t)nt; ++e) {
    const int32_t* v = &tri[4 * e];
    int32_t* o = &tri6[10 * e];
    for (int q = 0; q < 4; ++q) o[q] = v[q];
    for (int q = 0; q < 6; ++q) o[4 + q] = eid(v[TEDGES[q][0]], v[TEDGES[q][1]]);
  }
}

namespace {

// Cell box [i0,i1) x [j0,j1) x [k0,k1) of a region mesh; region 0 (fluid) has Gamma at
// K = 0, region 1 (porous) at K = 2 nz.
void make_problem3(Problem& P, const Mesh& m, int kind, int region, bool coarse, const int box[6], const int dbox[6]) {
  P.kind = kind; P.dim = 3; P.region = region; P.coarse = coarse;
  P.i0 = box[0]; P.i1 = box[1]; P.j0 = box[2]; P.j1 = box[3]; P.k0 = box[4]; P.k1 = box[5];
  P.di0 = dbox[0]; P.di1 = dbox[1]; P.dj0 = dbox[2]; P.dj1 = dbox[3]; P.dk0 = dbox[4]; P.dk1 = dbox[5];
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  P.touches_gamma = region == 0 ? (P.k0 == 0) : (P.k1 == nz);
  const int nI = 2 * (P.i1 - P.i0) + 1, nJ = 2 * (P.j1 - P.j0) + 1, nK = 2 * (P.k1 - P.k0) + 1;
  P.nn = nI * nJ * nK;
  P.gnode.resize(P.nn); P.nkind.resize(P.nn); P.art.resize(P.nn); P.inD.resize(P.nn);
  P.vidx.assign(P.nn, -1);
  P.vloc.clear();
  for (int c = 0; c < nK; ++c)
    for (int b = 0; b < nJ; ++b)
      for (int a = 0; a < nI; ++a) {
        const int l = a + nI * (b + nJ * c);
        const int I = 2 * P.i0 + a, J = 2 * P.j0 + b, K = 2 * P.k0 + c;
        P.gnode[l] = m.half_at3(I, J, K);
        const bool side = I == 0 || I == 2 * nx || J == 0 || J == 2 * ny;
        const bool region_bdry = side || (region == 0 ? K == 2 * nz : K == 0);
        const bool art = (I == 2 * P.i0 && P.i0 > 0) || (I == 2 * P.i1 && P.i1 < nx) ||
                         (J == 2 * P.j0 && P.j0 > 0) || (J == 2 * P.j1 && P.j1 < ny) ||
                         (K == 2 * P.k0 && P.k0 > 0) || (K == 2 * P.k1 && P.k1 < nz);
        P.art[l] = art;
        P.nkind[l] = region_bdry ? 1 : (art ? 2 : 0);
        P.inD[l] = I >= 2 * P.di0 && I <= 2 * P.di1 && J >= 2 * P.dj0 && J <= 2 * P.dj1 && K >= 2 * P.dk0 &&
                   K <= 2 * P.dk1;
        if (I % 2 == 0 && J % 2 == 0 && K % 2 == 0) {
          P.vidx[l] = (int)P.vloc.size();
          P.vloc.push_back(l);
        }
      }
  P.nvl = (int)P.vloc.size();
  P.etri.clear(); P.e6.clear(); P.e3.clear(); P.egam.clear();
  auto loc = [&](int I, int J, int K) { return (I - 2 * P.i0) + nI * ((J - 2 * P.j0) + nJ * (K - 2 * P.k0)); };
  for (int k = P.k0; k < P.k1; ++k)
    for (int j = P.j0; j < P.j1; ++j)
      for (int i = P.i0; i < P.i1; ++i) {
        const int cell = i + nx * (j + ny * k);
        for (int p = 0; p < 6; ++p) {
          int h[4][3];
          int c[3] = {2 * i, 2 * j, 2 * k};
          for (int d = 0; d < 3; ++d) h[0][d] = c[d];
          for (int s = 0; s < 3; ++s) {
            c[PERMS[p][s]] += 2;
            for (int d = 0; d < 3; ++d) h[1 + s][d] = c[d];
          }
          int nodes[10];
          for (int q = 0; q < 4; ++q) nodes[q] = loc(h[q][0], h[q][1], h[q][2]);
          for (int q = 0; q < 6; ++q) {
            const int* a = h[TEDGES[q][0]];
            const int* b = h[TEDGES[q][1]];
            nodes[4 + q] = loc((a[0] + b[0]) / 2, (a[1] + b[1]) / 2, (a[2] + b[2]) / 2);
          }
          P.etri.push_back(6 * cell + p);
          for (int q = 0; q < 10; ++q) P.e6.push_back(nodes[q]);
          for (int q = 0; q < 4; ++q) P.e3.push_back(P.vidx[nodes[q]]);
          // the face on Gamma: fluid bottom layer, tetrahedra whose first two steps stay in the
          // plane (perms (0,1,2), (1,0,2)): face v0 v1 v2, opposite v3; porous top layer,
          // first step along z (perms (2,0,1), (2,1,0)): face v1 v2 v3, opposite v0
          int8_t code = -1;
          if (region == 0 && k == 0 && PERMS[p][2] == 2) code = 3;
          if (region == 1 && k == nz - 1 && PERMS[p][0] == 2) code = 0;
          P.egam.push_back(code);
        }
      }
  P.ne = (int)P.etri.size();
  for (int e = 0; e < P.ne; ++e)
    for (int q = 0; q < 10; ++q)
      if (P.gnode[P.e6[10 * (size_t)e + q]] != m.tri6[10 * (size_t)P.etri[e] + q])
        std::fprintf(stderr, "tpns: internal 3D numbering mismatch\n");
}

void p2_tet_values(double x, double y, double z, double* N) {
  const double l[4] = {1 - x - y - z, x, y, z};
  for (int i = 0; i < 4; ++i) N[i] = l[i] * (2 * l[i] - 1);
  for (int q = 0; q < 6; ++q) N[4 + q] = 4 * l[TEDGES[q][0]] * l[TEDGES[q][1]];
}

// Fine nodal interpolant of coarse P2 (nb = 10) or P1 (nb = 4) functions: each fine point
// is located in its coarse cell and in the first of the cell's six tetrahedra whose
// barycentric coordinates are all >= -1e-12.
void prolong_table3(const Mesh& H, const double* pts, int npts, int nb, std::vector<int32_t>& idx,
                    std::vector<double>& w) {
  idx.resize((size_t)npts * nb);
  w.resize((size_t)npts * nb);
  auto cell_of = [](const std::vector<double>& g, int n, double x) {
    int c = (int)(std::upper_bound(g.begin(), g.end(), x) - g.begin()) - 1;
    return std::min(std::max(c, 0), n - 1);
  };
  for (int p = 0; p < npts; ++p) {
    const double x = pts[3 * (size_t)p], y = pts[3 * (size_t)p + 1], z = pts[3 * (size_t)p + 2];
    const int cell = cell_of(H.xs, H.nx, x) + H.nx * (cell_of(H.ys, H.ny, y) + H.ny * cell_of(H.zs, H.nz, z));
    for (int t = 0; t < 6; ++t) {
      const int tet = 6 * cell + t;
      const int32_t* v = &H.tri[4 * (size_t)tet];
      double a[3], J[3][3];
      for (int c = 0; c < 3; ++c) {
        a[c] = H.node[3 * (size_t)v[0] + c];
        for (int r = 0; r < 3; ++r) J[c][r] = H.node[3 * (size_t)v[1 + r] + c] - a[c];
      }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      double inv[3][3];
      inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
      inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
      inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
      inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      const double d[3] = {x - a[0], y - a[1], z - a[2]};
      double xi[3];
      for (int r = 0; r < 3; ++r) xi[r] = inv[r][0] * d[0] + inv[r][1] * d[1] + inv[r][2] * d[2];
      const double lmin = std::min(std::min(1 - xi[0] - xi[1] - xi[2], xi[0]), std::min(xi[1], xi[2]));
      if (lmin < -1e-12 && t < 5) continue;
      double N[10];
      if (nb == 10) {
        p2_tet_values(xi[0], xi[1], xi[2], N);
        for (int k = 0; k < 10; ++k) {
          idx[(size_t)p * 10 + k] = H.tri6[10 * (size_t)tet + k];
          w[(size_t)p * 10 + k] = std::fabs(N[k]) < 1e-15 ? 0.0 : N[k];
        }
      } else {
        N[0] = 1 - xi[0] - xi[1] - xi[2]; N[1] = xi[0]; N[2] = xi[1]; N[3] = xi[2];
        for (int k = 0; k < 4; ++k) {
          idx[(size_t)p * 4 + k] = v[k];
          w[(size_t)p * 4 + k] = std::fabs(N[k]) < 1e-15 ? 0.0 : N[k];
        }
      }
      break;
    }
  }
}

// Gamma partner nodes: the node of the other region's Gamma plane with the same (I, J).
void gam3(Problem& P, const Mesh& self, const Mesh& other, int region) {
  P.gam_src.assign(P.nn, -1);
  const int nI = 2 * (P.i1 - P.i0) + 1, nJ = 2 * (P.j1 - P.j0) + 1;
  const int Kg = region == 0 ? 0 : 2 * self.nz;
  const int Ko = region == 0 ? 2 * other.nz : 0;
  for (int l = 0; l < P.nn; ++l) {
    const int I = 2 * P.i0 + l % nI, J = 2 * P.j0 + (l / nI) % nJ, K = 2 * P.k0 + l / (nI * nJ);
    if (K == Kg) P.gam_src[l] = other.half_at3(I, J, Ko);
  }
}

}  // namespace

std::string build_layout3(const tpns_mesh_desc& md, const tpns_partition_desc& pd, Layout& L, int mf_leaf, int rank,
                          int nranks) {
  const int nc = md.nx_coarse, r = md.fine_per_coarse_x;
  if (nc <= 0 || r <= 0 || md.ny_coarse != nc) return "3D mesh: nx_coarse = ny_coarse > 0 and fine_per_coarse_x > 0";
  if (pd.nsub_x <= 0 || pd.nsub_y <= 0 || pd.nsub_z <= 0 || nc % pd.nsub_x || nc % pd.nsub_y || nc % pd.nsub_z ||
      pd.overlap < 0)
    return "subdomains must split the coarse cells evenly";
  L.dim = 3;
  std::vector<double> xH, xh, zcH, zch, zpH, zph;
  for (int i = 0; i <= nc; ++i) xH.push_back((double)i / (double)nc);
  for (int k = 0; k <= nc * r; ++k) xh.push_back((double)k / (double)(nc * r));
  for (double v : xH) { zcH.push_back(1.0 + v); zpH.push_back(v); }
  for (double v : xh) { zch.push_back(1.0 + v); zph.push_back(v); }
  L.mcH.build3(xH, xH, zcH);
  L.mch.build3(xh, xh, zch);
  L.mpH.build3(xH, xH, zpH);
  L.mph.build3(xh, xh, zph);
  const int n = nc * r;
  const int ns[3] = {pd.nsub_x, pd.nsub_y, pd.nsub_z};
  // local problems (independent of each other: built on host threads, kept in subdomain order)
  struct Sub {
    int region, box[6], dbox[6];
  };
  std::vector<Sub> subs;
  for (int region = 0; region < 2; ++region)
    for (int c = 0; c < ns[2]; ++c)
      for (int b = 0; b < ns[1]; ++b)
        for (int a = 0; a < ns[0]; ++a) {
          const int idx[3] = {a, b, c};
          Sub u;
          u.region = region;
          for (int d = 0; d < 3; ++d) {
            const int lo = idx[d] * n / ns[d], hi = (idx[d] + 1) * n / ns[d];
            u.dbox[2 * d] = lo;
            u.dbox[2 * d + 1] = hi;
            u.box[2 * d] = std::max(lo - pd.overlap, 0);
            u.box[2 * d + 1] = std::min(hi + pd.overlap, n);
          }
          subs.push_back(u);
        }
  std::vector<Problem> probs(subs.size());
  std::vector<std::string> errs(subs.size());
  parallel_for((int)subs.size(), [&](int i) {
    const Sub& u = subs[i];
    try {
      make_problem3(probs[i], u.region == 0 ? L.mch : L.mph, u.region == 0 ? PK_OSEEN : PK_DARCY, u.region, false,
                    u.box, u.dbox);
    } catch (...) {
      errs[i] = "host layout of a local problem failed";
      return;
    }
    errs[i] = finish_local_problem(probs[i], mf_leaf);
  });
  for (const std::string& e : errs)
    if (!e.empty()) return e;
  L.fluid.clear();
  L.porous.clear();
  for (size_t i = 0; i < subs.size(); ++i) (subs[i].region == 0 ? L.fluid : L.porous).push_back(std::move(probs[i]));
  const int whole[6] = {0, nc, 0, nc, 0, nc};
  make_problem3(L.cfl, L.mcH, PK_OSEEN, 0, true, whole, whole);
  if (!finish_problem(L.cfl)) return kLongRun;
  make_problem3(L.cpo, L.mpH, PK_DARCY, 1, true, whole, whole);
  if (!finish_problem(L.cpo)) return kLongRun;
  for (auto& P : L.fluid) gam3(P, L.mch, L.mph, 0);
  for (auto& P : L.porous) gam3(P, L.mph, L.mch, 1);
  gam3(L.cfl, L.mcH, L.mpH, 0);
  gam3(L.cpo, L.mpH, L.mcH, 1);
  prolong_table3(L.mcH, L.mch.node.data(), L.mch.nn, 10, L.pc2_idx, L.pc2_w);
  prolong_table3(L.mcH, L.mch.node.data(), L.mch.nv, 4, L.pc1_idx, L.pc1_w);
  prolong_table3(L.mpH, L.mph.node.data(), L.mph.nn, 10, L.pp2_idx, L.pp2_w);
  glue_table(L.fluid, L.mch.nn, false, L.gc_ptr, L.gc_prob, L.gc_node, L.gc_w);
  glue_table(L.porous, L.mph.nn, false, L.gp_ptr, L.gp_prob, L.gp_node, L.gp_w);
  glue_table(L.fluid, L.mch.nv, true, L.gv_ptr, L.gv_prob, L.gv_vert, L.gv_w);
  for (int i = 0; i < L.mch.nn; ++i)
    if (L.gc_ptr[i + 1] == L.gc_ptr[i]) return "a conduit node is in no D_j";
  for (int i = 0; i < L.mph.nn; ++i)
    if (L.gp_ptr[i + 1] == L.gp_ptr[i]) return "a porous node is in no D_j";
  return split_ranks(L, rank, nranks);
}

// ------------------------------------------------------------------------------ 3D reference tables
namespace {

// 3-point Gauss rule on [0,1] for the weight (1-u)^alpha: nodes are the roots of the monic
// cubic orthogonal to 1, u, u^2 under that weight (moments m_k = k! alpha! / (k+alpha+1)!),
// weights from the moment equations; computed in long double and rounded once.
void gauss_jacobi3(int alpha, double* x, double* w) {
  typedef long double R;
  auto fact = [](int k) { R f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
  R m[6];
  for (int k = 0; k < 6; ++k) m[k] = fact(k) * fact(alpha) / fact(k + alpha + 1);
  // c0 m_i + c1 m_{i+1} + c2 m_{i+2} = -m_{i+3}, i = 0, 1, 2
  R A[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) A[i][j] = m[i + j];
    A[i][3] = -m[i + 3];
  }
  for (int c = 0; c < 3; ++c) {
    int pv = c;
    for (int i = c + 1; i < 3; ++i)
      if (std::fabs((double)A[i][c]) > std::fabs((double)A[pv][c])) pv = i;
    for (int j = 0; j < 4; ++j) std::swap(A[c][j], A[pv][j]);
    for (int i = 0; i < 3; ++i) {
      if (i == c) continue;
      const R f = A[i][c] / A[c][c];
      for (int j = c; j < 4; ++j) A[i][j] -= f * A[c][j];
    }
  }
  const R c0 = A[0][3] / A[0][0], c1 = A[1][3] / A[1][1], c2 = A[2][3] / A[2][2];
  auto p = [&](R u) { return ((u + c2) * u + c1) * u + c0; };
  auto dp = [&](R u) { return (3 * u + 2 * c2) * u + c1; };
  // the roots are simple and lie in (0, 1): bracket them on a fine grid, then Newton
  R roots[3];
  int nr = 0;
  const int G = 4096;
  for (int g = 0; g < G && nr < 3; ++g) {
    R a = (R)g / G, b = (R)(g + 1) / G;
    if (p(a) == 0) { roots[nr++] = a; continue; }
    if (p(a) * p(b) < 0) {
      R u = 0.5L * (a + b);
      for (int it = 0; it < 60; ++it) {
        R du = p(u) / dp(u);
        u -= du;
        if (std::fabs((double)du) < 1e-30) break;
      }
      roots[nr++] = u;
    }
  }
  // weights: sum_i w_i u_i^k = m_k, k = 0, 1, 2 (Lagrange form)
  for (int i = 0; i < 3; ++i) {
    const R a = roots[(i + 1) % 3], b = roots[(i + 2) % 3];
    // int l_i (1-u)^alpha with l_i = (u - a)(u - b) / ((u_i - a)(u_i - b))
    const R num = m[2] - (a + b) * m[1] + a * b * m[0];
    w[i] = (double)(num / ((roots[i] - a) * (roots[i] - b)));
    x[i] = (double)roots[i];
  }
}

void p2_tet_grads(double x, double y, double z, double dN[10][3]) {
  const double l[4] = {1 - x - y - z, x, y, z};
  const double dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int i = 0; i < 4; ++i)
    for (int r = 0; r < 3; ++r) dN[i][r] = (4 * l[i] - 1) * dl[i][r];
  for (int q = 0; q < 6; ++q) {
    const int a = TEDGES[q][0], b = TEDGES[q][1];
    for (int r = 0; r < 3; ++r) dN[4 + q][r] = 4 * (l[a] * dl[b][r] + l[b] * dl[a][r]);
  }
}

}  // namespace

void build_ref_tables3(RefTables3& R) {
  double u[3], wu[3], v[3], wv[3], s[3], ws[3];
  gauss_jacobi3(2, u, wu);
  gauss_jacobi3(1, v, wv);
  gauss_jacobi3(0, s, ws);
  double N[27][10], D[27][10][3], Q[27][4], W[27];
  int q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c, ++q) {
        const double x = u[a], y = v[b] * (1.0 - u[a]), z = s[c] * (1.0 - u[a]) * (1.0 - v[b]);
        R.qp[q][0] = x; R.qp[q][1] = y; R.qp[q][2] = z;
        W[q] = wu[a] * wv[b] * ws[c];
        R.qw[q] = W[q];
        p2_tet_values(x, y, z, N[q]);
        p2_tet_grads(x, y, z, D[q]);
        Q[q][0] = 1 - x - y - z; Q[q][1] = x; Q[q][2] = y; Q[q][3] = z;
        for (int i = 0; i < 10; ++i) R.qphi[q][i] = N[q][i];
      }
  std::fill(&R.M[0][0], &R.M[0][0] + 100, 0.0);
  std::fill(&R.S[0][0][0][0], &R.S[0][0][0][0] + 900, 0.0);
  std::fill(&R.T[0][0][0][0], &R.T[0][0][0][0] + 3000, 0.0);
  std::fill(&R.U[0][0][0][0], &R.U[0][0][0][0] + 3000, 0.0);
  std::fill(&R.B[0][0][0], &R.B[0][0][0] + 120, 0.0);
  for (q = 0; q < 27; ++q)
    for (int i = 0; i < 10; ++i) {
      for (int j = 0; j < 10; ++j) {
        R.M[i][j] += W[q] * N[q][i] * N[q][j];
        for (int r = 0; r < 3; ++r)
          for (int t = 0; t < 3; ++t) R.S[i][j][r][t] += W[q] * D[q][i][r] * D[q][j][t];
        for (int k = 0; k < 10; ++k)
          for (int r = 0; r < 3; ++r) {
            R.T[k][j][i][r] += W[q] * N[q][k] * D[q][j][r] * N[q][i];
            R.U[i][j][k][r] += W[q] * N[q][i] * N[q][j] * D[q][k][r];
          }
      }
      for (int k = 0; k < 4; ++k)
        for (int r = 0; r < 3; ++r) R.B[k][i][r] += W[q] * Q[q][k] * D[q][i][r];
    }
  // faces: the 7-point degree-5 triangle rule (Radon), P2 basis (v0, v1, v2, m01, m02, m12)
  const double s15 = std::sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
  const double w1 = (155.0 - s15) / 2400.0, w2 = (155.0 + s15) / 2400.0;
  const double P[7][2] = {{1.0 / 3.0, 1.0 / 3.0}, {a1, a1}, {1.0 - 2.0 * a1, a1}, {a1, 1.0 - 2.0 * a1},
                          {a2, a2}, {1.0 - 2.0 * a2, a2}, {a2, 1.0 - 2.0 * a2}};
  const double FW[7] = {9.0 / 80.0, w1, w1, w1, w2, w2, w2};
  const int FE[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (q = 0; q < 7; ++q) {
    const double x = P[q][0], y = P[q][1];
    R.fqp[q][0] = x; R.fqp[q][1] = y; R.fqw[q] = FW[q];
    const double l[3] = {1 - x - y, x, y};
    const double dl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
    for (int i = 0; i < 3; ++i) {
      R.fphi[q][i] = l[i] * (2 * l[i] - 1);
      for (int r = 0; r < 2; ++r) R.fdphi[q][i][r] = (4 * l[i] - 1) * dl[i][r];
    }
    for (int k = 0; k < 3; ++k) {
      const int a = FE[k][0], b = FE[k][1];
      R.fphi[q][3 + k] = 4 * l[a] * l[b];
      for (int r = 0; r < 2; ++r) R.fdphi[q][3 + k][r] = 4 * (l[a] * dl[b][r] + l[b] * dl[a][r]);
    }
  }
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double m = 0.0;
      for (q = 0; q < 7; ++q) m += FW[q] * R.fphi[q][a] * R.fphi[q][b];
      R.fM[a][b] = m;
    }
}

}  // namespace tpns
