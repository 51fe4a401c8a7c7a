// Host-side layout of the local parallel two-grid method: meshes of both regions on both
// levels, overlapping subdomains (Algorithm 3, Step 2), band orderings, CSR patterns,
// sorted element-to-CSR scatter maps packed in warp-sized chunks, prolongation and glue
// tables.  Pure host code; results are uploaded once by the context.
#include "setup.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <map>
#include <numeric>
#include <thread>
#include <tuple>

namespace tpns {

void Mesh::build(const std::vector<double>& xs_, const std::vector<double>& ys_) {
  xs = xs_;
  ys = ys_;
  nx = (int)xs.size() - 1;
  ny = (int)ys.size() - 1;
  nv = (nx + 1) * (ny + 1);
  nt = 2 * nx * ny;
  auto vid = [&](int i, int j) { return i + (nx + 1) * j; };
  tri.resize((size_t)nt * 3);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)i + (size_t)nx * j;
      int32_t* lo = &tri[6 * c];
      lo[0] = vid(i, j); lo[1] = vid(i + 1, j); lo[2] = vid(i + 1, j + 1);
      lo[3] = vid(i, j); lo[4] = vid(i + 1, j + 1); lo[5] = vid(i, j + 1);
    }
  // edges of the grid: horizontal, vertical and diagonal, ordered by (min vid, max vid)
  std::vector<std::pair<int32_t, int32_t>> edges;
  edges.reserve((size_t)3 * nx * ny + nx + ny);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (i < nx) edges.push_back({vid(i, j), vid(i + 1, j)});
      if (j < ny) edges.push_back({vid(i, j), vid(i, j + 1)});
      if (i < nx && j < ny) edges.push_back({vid(i, j), vid(i + 1, j + 1)});
    }
  std::sort(edges.begin(), edges.end());
  nedge = (int)edges.size();
  nn = nv + nedge;
  auto eid = [&](int32_t a, int32_t b) {
    std::pair<int32_t, int32_t> k{std::min(a, b), std::max(a, b)};
    auto it = std::lower_bound(edges.begin(), edges.end(), k);
    return nv + (int32_t)(it - edges.begin());
  };
  node.resize((size_t)nn * 2);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      node[2 * (size_t)vid(i, j)] = xs[i];
      node[2 * (size_t)vid(i, j) + 1] = ys[j];
    }
  for (int e = 0; e < nedge; ++e) {
    int a = edges[e].first, b = edges[e].second;
    node[2 * (size_t)(nv + e)] = 0.5 * (node[2 * (size_t)a] + node[2 * (size_t)b]);
    node[2 * (size_t)(nv + e) + 1] = 0.5 * (node[2 * (size_t)a + 1] + node[2 * (size_t)b + 1]);
  }
  tri6.resize((size_t)nt * 6);
  for (int t = 0; t < nt; ++t) {
    int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    int32_t* o = &tri6[6 * (size_t)t];
    o[0] = a; o[1] = b; o[2] = c;
    o[3] = eid(a, b); o[4] = eid(b, c); o[5] = eid(c, a);
  }
  half.assign((size_t)(2 * ny + 1) * (2 * nx + 1), -1);
  auto H = [&](int I, int J) -> int32_t& { return half[(size_t)J * (2 * nx + 1) + I]; };
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      H(2 * i, 2 * j) = vid(i, j);
      if (i < nx) H(2 * i + 1, 2 * j) = eid(vid(i, j), vid(i + 1, j));
      if (j < ny) H(2 * i, 2 * j + 1) = eid(vid(i, j), vid(i, j + 1));
      if (i < nx && j < ny) H(2 * i + 1, 2 * j + 1) = eid(vid(i, j), vid(i + 1, j + 1));
    }
}

// ------------------------------------------------------------------------------ breaks
struct Breaks {
  std::vector<double> xs_H, xs_h, ysc_H, ysc_h, ysp_H, ysp_h;
  std::vector<int> fy_c, fy_p;   // fine row index of every coarse line
  std::vector<int> fx;
};

static Breaks make_breaks(const tpns_mesh_desc& md) {
  Breaks b;
  int nxc = md.nx_coarse, nyc = md.ny_coarse, r = md.fine_per_coarse_x;
  for (int i = 0; i <= nxc; ++i) b.xs_H.push_back((double)i / (double)nxc);
  for (int k = 0; k <= nxc * r; ++k) b.xs_h.push_back((double)k / (double)(nxc * r));
  for (int i = 0; i <= nxc; ++i) b.fx.push_back(i * r);
  // conduit: coarse row c lies at distance c from Gamma
  b.ysc_h.push_back(1.0);
  b.fy_c.push_back(0);
  for (int c = 0; c < nyc; ++c) {
    int m = md.fine_rows_from_gamma[c];
    for (int k = 1; k <= m; ++k) b.ysc_h.push_back(1.0 + (double)(c * m + k) / (double)(nyc * m));
    b.fy_c.push_back(b.fy_c.back() + m);
  }
  for (int c = 0; c <= nyc; ++c) b.ysc_H.push_back(1.0 + (double)c / (double)nyc);
  // porous: coarse row c (from y = 0) lies at distance nyc-1-c from Gamma
  b.ysp_h.push_back(0.0);
  b.fy_p.push_back(0);
  for (int c = 0; c < nyc; ++c) {
    int m = md.fine_rows_from_gamma[nyc - 1 - c];
    for (int k = 1; k <= m; ++k) b.ysp_h.push_back((double)(c * m + k) / (double)(nyc * m));
    b.fy_p.push_back(b.fy_p.back() + m);
  }
  for (int c = 0; c <= nyc; ++c) b.ysp_H.push_back((double)c / (double)nyc);
  return b;
}

// ------------------------------------------------------------------------------ problems
// Cell box [i0,i1) x [j0,j1) of a region mesh; region 0 has Gamma at J = 0, region 1 at
// J = 2 ny.  `whole` = coarse whole-region problem (no artificial boundary).
static void make_problem(Problem& P, const Mesh& m, int kind, int region, bool coarse,
                         int i0, int i1, int j0, int j1, int di0, int di1, int dj0, int dj1) {
  P.kind = kind; P.region = region; P.coarse = coarse;
  P.i0 = i0; P.i1 = i1; P.j0 = j0; P.j1 = j1;
  P.di0 = di0; P.di1 = di1; P.dj0 = dj0; P.dj1 = dj1;
  const int nx = m.nx, ny = m.ny;
  const int gJ = region == 0 ? 0 : 2 * ny;
  P.touches_gamma = region == 0 ? (j0 == 0) : (j1 == ny);
  const int nI = 2 * (i1 - i0) + 1, nJ = 2 * (j1 - j0) + 1;
  P.nn = nI * nJ;
  P.gnode.resize(P.nn); P.nkind.resize(P.nn); P.art.resize(P.nn); P.inD.resize(P.nn);
  P.vidx.assign(P.nn, -1);
  P.vloc.clear();
  for (int b = 0; b < nJ; ++b)
    for (int a = 0; a < nI; ++a) {
      int l = a + nI * b;
      int I = 2 * i0 + a, J = 2 * j0 + b;
      P.gnode[l] = m.half_at(I, J);
      bool region_bdry = region == 0 ? (I == 0 || I == 2 * nx || J == 2 * ny)
                                     : (I == 0 || I == 2 * nx || J == 0);
      bool art = (I == 2 * i0 && i0 > 0) || (I == 2 * i1 && i1 < nx) ||
                 (J == 2 * j0 && j0 > 0) || (J == 2 * j1 && j1 < ny);
      P.art[l] = art;
      P.nkind[l] = region_bdry ? 1 : (art ? 2 : 0);
      P.inD[l] = (I >= 2 * di0 && I <= 2 * di1 && J >= 2 * dj0 && J <= 2 * dj1);
      if (I % 2 == 0 && J % 2 == 0) {
        P.vidx[l] = (int)P.vloc.size();
        P.vloc.push_back(l);
      }
    }
  P.nvl = (int)P.vloc.size();
  (void)gJ;
  // elements of the box, mesh order
  P.etri.clear(); P.e6.clear(); P.e3.clear(); P.egam.clear();
  auto loc = [&](int I, int J) { return (I - 2 * i0) + nI * (J - 2 * j0); };
  for (int j = j0; j < j1; ++j)
    for (int i = i0; i < i1; ++i) {
      int c = i + nx * j;
      // local node ids of the two triangles from half-grid positions
      int v00 = loc(2 * i, 2 * j), v10 = loc(2 * i + 2, 2 * j), v11 = loc(2 * i + 2, 2 * j + 2),
          v01 = loc(2 * i, 2 * j + 2);
      int mb = loc(2 * i + 1, 2 * j), mr = loc(2 * i + 2, 2 * j + 1), md = loc(2 * i + 1, 2 * j + 1),
          ml = loc(2 * i, 2 * j + 1), mt = loc(2 * i + 1, 2 * j + 2);
      int lower[6] = {v00, v10, v11, mb, mr, md};
      int upper[6] = {v00, v11, v01, md, mt, ml};
      for (int t = 0; t < 2; ++t) {
        const int* s = t == 0 ? lower : upper;
        P.etri.push_back(2 * c + t);
        for (int k = 0; k < 6; ++k) P.e6.push_back(s[k]);
        for (int k = 0; k < 3; ++k) P.e3.push_back(P.vidx[s[k]]);
        int8_t code = -1;
        if (region == 0 && t == 0 && j == 0) code = 0;        // bottom edge v00-v10 on Gamma
        if (region == 1 && t == 1 && j == ny - 1) code = 1;   // top edge v01-v11 on Gamma
        P.egam.push_back(code);
      }
    }
  P.ne = (int)P.etri.size();
  // sanity: element nodes agree with the mesh's own numbering
  for (int e = 0; e < P.ne; ++e)
    for (int k = 0; k < 6; ++k)
      if (P.gnode[P.e6[6 * e + k]] != m.tri6[6 * (size_t)P.etri[e] + k]) {
        std::fprintf(stderr, "tpns: internal numbering mismatch\n");
      }
}

// Unknowns in band order.  Sweep along the longer side of the box; key of a velocity
// unknown (col, 0, row, comp), of a vertex pressure (col + 1, 1, row, 0): each pressure
// follows the velocities of the next half-grid column, so that every leading block of
// the saddle-point matrix is invertible and the LU needs no pivoting.
// 3D: the sweep runs along the longest side of the box; "column" is then a plane of the half
// grid and every vertex pressure follows the velocities of the next plane.
static void order_unknowns(Problem& P) {
  const int D = P.dim;
  const int nI = 2 * (P.i1 - P.i0) + 1, nJ = 2 * (P.j1 - P.j0) + 1, nK = 2 * (P.k1 - P.k0) + 1;
  const int ext[3] = {P.i1 - P.i0, P.j1 - P.j0, P.k1 - P.k0};
  int axis = 0;
  if (D == 2) {
    axis = ext[0] >= ext[1] ? 0 : 1;
  } else {
    for (int d = 1; d < 3; ++d)
      if (ext[d] > ext[axis]) axis = d;
  }
  const int PC = D;   // component index of the pressure
  struct Key { int a, b, c, d, node, comp; };
  std::vector<Key> keys;
  for (int l = 0; l < P.nn; ++l) {
    int crd[3] = {l % nI, (l / nI) % nJ, D == 3 ? l / (nI * nJ) : 0};
    int col = crd[axis], row;
    if (D == 2) {
      row = axis == 0 ? crd[1] : crd[0];
    } else {
      const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
      const int n1 = o1 == 0 ? nI : nJ;
      row = crd[o2] * n1 + crd[o1];
    }
    (void)nK;
    if (P.nkind[l] == 0) {
      if (P.kind == PK_OSEEN) {
        for (int c = 0; c < D; ++c) keys.push_back({col, 0, row, c, l, c});
      } else {
        keys.push_back({col, 0, row, 0, l, 0});
      }
    }
    if (P.kind == PK_OSEEN && P.vidx[l] >= 0 && !P.art[l]) keys.push_back({col + 1, 1, row, 0, l, PC});
  }
  std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
    return std::tie(x.a, x.b, x.c, x.d) < std::tie(y.a, y.b, y.c, y.d);
  });
  P.n = (int)keys.size();
  P.dof_node.resize(P.n); P.dof_comp.resize(P.n);
  if (P.kind == PK_OSEEN) {
    P.node_dof.assign((size_t)D * P.nn, -1);
    P.vert_dof.assign(P.nvl, -1);
  } else {
    P.node_dof.assign(P.nn, -1);
    P.vert_dof.clear();
  }
  for (int d = 0; d < P.n; ++d) {
    P.dof_node[d] = keys[d].node;
    P.dof_comp[d] = keys[d].comp;
    if (P.kind == PK_OSEEN) {
      if (keys[d].comp < D) P.node_dof[(size_t)D * keys[d].node + keys[d].comp] = d;
      else P.vert_dof[P.vidx[keys[d].node]] = d;
    } else {
      P.node_dof[keys[d].node] = d;
    }
  }
  const int S = P.slots(), NPE = P.npe(), VPE = P.vpe(), VS = P.vslots();
  P.slot_dof.assign((size_t)P.ne * S, -1);
  for (int e = 0; e < P.ne; ++e) {
    if (P.kind == PK_OSEEN) {
      for (int i = 0; i < NPE; ++i)
        for (int a = 0; a < D; ++a)
          P.slot_dof[(size_t)e * S + D * i + a] = P.node_dof[(size_t)D * P.e6[(size_t)NPE * e + i] + a];
      for (int k = 0; k < VPE; ++k) P.slot_dof[(size_t)e * S + VS + k] = P.vert_dof[P.e3[(size_t)VPE * e + k]];
    } else {
      for (int i = 0; i < NPE; ++i) P.slot_dof[(size_t)e * S + i] = P.node_dof[P.e6[(size_t)NPE * e + i]];
    }
  }
}

// Pack (target, source) contributions sorted by target into warp chunks of 32 lanes so
// that no run of equal targets straddles two chunks (padding lanes get target -1).  The
// segmented warp reduction adds one run inside one warp, so a target with more than 32
// contributions cannot be packed: returns false (nothing is truncated).
static bool pack_chunks(std::vector<std::pair<int32_t, int32_t>>& c, std::vector<int32_t>& tgt,
                        std::vector<int32_t>& src) {
  std::sort(c.begin(), c.end());
  tgt.clear(); src.clear();
  size_t i = 0;
  int lane = 0;
  while (i < c.size()) {
    size_t j = i;
    while (j < c.size() && c[j].first == c[i].first) ++j;
    int len = (int)(j - i);
    if (len > 32) return false;
    if (lane + len > 32) {
      while (lane < 32) { tgt.push_back(-1); src.push_back(0); ++lane; }
      lane = 0;
    }
    for (size_t k = i; k < j; ++k) { tgt.push_back(c[k].first); src.push_back(c[k].second); }
    lane += len;
    if (lane == 32) lane = 0;
    i = j;
  }
  while (lane != 0 && lane < 32) { tgt.push_back(-1); src.push_back(0); ++lane; }
  return true;
}

static bool build_pattern(Problem& P) {
  const int S = P.slots(), VS = P.vslots();
  std::vector<std::vector<int32_t>> rows(P.n);
  for (int e = 0; e < P.ne; ++e)
    for (int r = 0; r < S; ++r) {
      int dr = P.slot_dof[(size_t)e * S + r];
      if (dr < 0) continue;
      for (int c = 0; c < S; ++c) {
        int dc = P.slot_dof[(size_t)e * S + c];
        if (dc < 0) continue;
        if (P.kind == PK_OSEEN && r >= VS && c >= VS) continue;   // zero pressure block
        rows[dr].push_back(dc);
      }
    }
  P.rowptr.assign(P.n + 1, 0);
  P.colidx.clear(); P.rowof.clear();
  P.kl = 0; P.ku = 0;
  for (int r = 0; r < P.n; ++r) {
    auto& v = rows[r];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    for (int c : v) {
      P.colidx.push_back(c);
      P.rowof.push_back(r);
      P.kl = std::max(P.kl, r - c);
      P.ku = std::max(P.ku, c - r);
    }
    P.rowptr[r + 1] = (int32_t)P.colidx.size();
  }
  // scatter maps
  std::vector<std::pair<int32_t, int32_t>> mc, rc;
  for (int e = 0; e < P.ne; ++e)
    for (int r = 0; r < S; ++r) {
      int dr = P.slot_dof[(size_t)e * S + r];
      if (dr < 0) continue;
      rc.push_back({dr, e * S + r});
      for (int c = 0; c < S; ++c) {
        int dc = P.slot_dof[(size_t)e * S + c];
        if (dc < 0) continue;
        if (P.kind == PK_OSEEN && r >= VS && c >= VS) continue;
        const int32_t* b = &P.colidx[P.rowptr[dr]];
        const int32_t* en = &P.colidx[P.rowptr[dr + 1]];
        int32_t k = P.rowptr[dr] + (int32_t)(std::lower_bound(b, en, dc) - b);
        mc.push_back({k, e * S * S + r * S + c});
      }
    }
  if (!pack_chunks(mc, P.mtgt, P.msrc) || !pack_chunks(rc, P.rtgt, P.rsrc)) return false;
  // algorithmic flops of the unpivoted band LU under this ordering
  double f = 0;
  for (int j = 0; j < P.n; ++j) {
    double l = std::min(P.kl, P.n - 1 - j), u = std::min(P.ku, P.n - 1 - j);
    f += l + 2.0 * l * u;
  }
  P.lu_flops = f;
  return true;
}

bool finish_problem(Problem& P) {
  order_unknowns(P);
  return build_pattern(P);
}

void parallel_for(int n, const std::function<void(int)>& task) {
  if (n <= 0) return;
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = std::min(n, (int)std::min(hw ? hw : 1u, 16u));
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) task(i);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(work);
    } catch (...) {
      break;   // the tasks left run on the threads already started and on this one
    }
  }
  work();
  for (auto& th : pool) th.join();
}

std::string finish_local_problem(Problem& P, int mf_leaf) {
  try {
    if (!finish_problem(P)) return kLongRun;
    return mf_leaf > 0 ? analyse_mf(P, mf_leaf) : std::string();
  } catch (const std::exception& e) {
    return std::string("host layout of a local problem failed: ") + e.what();
  } catch (...) {
    return "host layout of a local problem failed";
  }
}

const char* kLongRun = "a matrix or vector entry receives more than 32 element contributions";

// Multifrontal analysis of a local system (Oseen, or the pattern shared by the three Darcy
// fields): the unknowns' half-grid coordinates in the box (vertices at even coordinates) drive
// the nested dissection.
std::string analyse_mf(Problem& P, int leaf) {
  const int D = P.dim;
  const int nI = 2 * (P.i1 - P.i0) + 1, nJ = 2 * (P.j1 - P.j0) + 1;
  std::vector<int32_t> coord((size_t)P.n * D);
  std::vector<int8_t> pres(P.n);
  for (int d = 0; d < P.n; ++d) {
    const int l = P.dof_node[d];
    coord[(size_t)D * d] = l % nI;
    if (D == 2) {
      coord[(size_t)D * d + 1] = l / nI;
    } else {
      coord[(size_t)D * d + 1] = (l / nI) % nJ;
      coord[(size_t)D * d + 2] = l / (nI * nJ);
    }
    pres[d] = P.dof_comp[d] == D;
  }
  return mf_analyse(P.n, D, coord.data(), pres.data(), P.rowptr.data(), P.colidx.data(), leaf, P.mf);
}

// ------------------------------------------------------------------------------ prolongation
static void p2_values(double x, double y, double* N) {
  double l0 = 1 - x - y, l1 = x, l2 = y;
  N[0] = l0 * (2 * l0 - 1); N[1] = l1 * (2 * l1 - 1); N[2] = l2 * (2 * l2 - 1);
  N[3] = 4 * l0 * l1; N[4] = 4 * l1 * l2; N[5] = 4 * l2 * l0;
}

// Fine nodal interpolant of coarse P2 (nb = 6) or P1 (nb = 3) functions.
static void prolong_table(const Mesh& H, const double* pts, int npts, int nb,
                          std::vector<int32_t>& idx, std::vector<double>& w) {
  idx.resize((size_t)npts * nb);
  w.resize((size_t)npts * nb);
  for (int p = 0; p < npts; ++p) {
    double x = pts[2 * p], y = pts[2 * p + 1];
    int ci = (int)(std::upper_bound(H.xs.begin(), H.xs.end(), x) - H.xs.begin()) - 1;
    int cj = (int)(std::upper_bound(H.ys.begin(), H.ys.end(), y) - H.ys.begin()) - 1;
    ci = std::min(std::max(ci, 0), H.nx - 1);
    cj = std::min(std::max(cj, 0), H.ny - 1);
    bool done = false;
    for (int t = 0; t < 2 && !done; ++t) {
      int tr = 2 * (ci + H.nx * cj) + t;
      const int32_t* v = &H.tri[3 * (size_t)tr];
      double ax = H.node[2 * v[0]], ay = H.node[2 * v[0] + 1];
      double J00 = H.node[2 * v[1]] - ax, J10 = H.node[2 * v[1] + 1] - ay;
      double J01 = H.node[2 * v[2]] - ax, J11 = H.node[2 * v[2] + 1] - ay;
      double det = J00 * J11 - J01 * J10;
      double xi = (J11 * (x - ax) - J01 * (y - ay)) / det;
      double et = (-J10 * (x - ax) + J00 * (y - ay)) / det;
      double lmin = std::min(std::min(1 - xi - et, xi), et);
      if (lmin < -1e-12 && t == 0) continue;
      double N[6];
      if (nb == 6) {
        p2_values(xi, et, N);
        for (int k = 0; k < 6; ++k) {
          idx[(size_t)p * 6 + k] = H.tri6[6 * (size_t)tr + k];
          w[(size_t)p * 6 + k] = std::fabs(N[k]) < 1e-15 ? 0.0 : N[k];
        }
      } else {
        N[0] = 1 - xi - et; N[1] = xi; N[2] = et;
        for (int k = 0; k < 3; ++k) {
          idx[(size_t)p * 3 + k] = v[k];
          w[(size_t)p * 3 + k] = std::fabs(N[k]) < 1e-15 ? 0.0 : N[k];
        }
      }
      done = true;
    }
  }
}

void glue_table(const std::vector<Problem>& probs, int nnodes, bool vertices,
                std::vector<int32_t>& ptr, std::vector<int32_t>& prob,
                std::vector<int32_t>& loc, std::vector<double>& w) {
  std::vector<std::vector<std::pair<int32_t, int32_t>>> lists(nnodes);
  for (size_t p = 0; p < probs.size(); ++p) {
    const Problem& P = probs[p];
    if (!vertices) {
      for (int l = 0; l < P.nn; ++l)
        if (P.inD[l]) lists[P.gnode[l]].push_back({(int32_t)p, l});
    } else {
      for (int v = 0; v < P.nvl; ++v) {
        int l = P.vloc[v];
        if (P.inD[l]) lists[P.gnode[l]].push_back({(int32_t)p, v});
      }
    }
  }
  ptr.assign(nnodes + 1, 0);
  prob.clear(); loc.clear(); w.clear();
  for (int i = 0; i < nnodes; ++i) {
    for (auto& pr : lists[i]) {
      prob.push_back(pr.first);
      loc.push_back(pr.second);
      w.push_back(1.0 / (double)lists[i].size());
    }
    ptr[i + 1] = (int32_t)prob.size();
  }
}

// Indices of the problems a rank keeps: estimated per-step work of each problem, largest
// first, each to the least loaded rank (ties to the lower rank).
static std::vector<int> owned(const std::vector<Problem>& list, int rank, int nranks) {
  std::vector<std::pair<double, int>> w;
  for (int i = 0; i < (int)list.size(); ++i) {
    const Problem& P = list[i];
    double entries = P.mf.fronts.empty() ? (double)P.n * (P.kl + P.ku + 1) : P.mf.factor_entries;
    double work = P.kind == PK_OSEEN ? (P.mf.fronts.empty() ? P.lu_flops : P.mf.flops) + 6.0 * entries
                                     : 18.0 * entries;   // three fields, about three solve passes
    w.push_back({-work, i});
  }
  std::sort(w.begin(), w.end());
  std::vector<double> load(nranks, 0.0);
  std::vector<int> mine;
  for (auto& e : w) {
    int r = 0;
    for (int k = 1; k < nranks; ++k)
      if (load[k] < load[r]) r = k;
    load[r] += -e.first;
    if (r == rank) mine.push_back(e.second);
  }
  std::sort(mine.begin(), mine.end());
  return mine;
}

// Keep the glue entries of the kept problems (renumbered), with their weights unchanged.
static void filter_glue(std::vector<int32_t>& ptr, std::vector<int32_t>& prob, std::vector<int32_t>& loc,
                        std::vector<double>& w, const std::vector<int>& remap) {
  std::vector<int32_t> p2(ptr.size(), 0), pr2, lo2;
  std::vector<double> w2;
  for (size_t i = 0; i + 1 < ptr.size(); ++i) {
    for (int k = ptr[i]; k < ptr[i + 1]; ++k)
      if (remap[prob[k]] >= 0) {
        pr2.push_back(remap[prob[k]]);
        lo2.push_back(loc[k]);
        w2.push_back(w[k]);
      }
    p2[i + 1] = (int32_t)pr2.size();
  }
  ptr.swap(p2);
  prob.swap(pr2);
  loc.swap(lo2);
  w.swap(w2);
}

std::string build_layout(const tpns_mesh_desc& md, const tpns_partition_desc& pd, Layout& L, int mf_leaf,
                         int rank, int nranks) {
  if (md.dim == 3) return build_layout3(md, pd, L, mf_leaf, rank, nranks);
  if (md.dim != 0 && md.dim != 2) return "invalid mesh dimension";
  if (md.nx_coarse <= 0 || md.ny_coarse <= 0 || md.ny_coarse > TPNS_MAX_COARSE_ROWS ||
      md.fine_per_coarse_x <= 0)
    return "invalid mesh description";
  for (int c = 0; c < md.ny_coarse; ++c)
    if (md.fine_rows_from_gamma[c] <= 0) return "invalid fine row count";
  if (pd.nsub_x <= 0 || pd.nsub_y <= 0 || md.nx_coarse % pd.nsub_x || md.ny_coarse % pd.nsub_y ||
      pd.overlap < 0)
    return "subdomains must split the coarse cells evenly";
  Breaks b = make_breaks(md);
  L.mcH.build(b.xs_H, b.ysc_H);
  L.mch.build(b.xs_h, b.ysc_h);
  L.mpH.build(b.xs_H, b.ysp_H);
  L.mph.build(b.xs_h, b.ysp_h);
  // local problems (Algorithm 3 Step 2), same layout in both regions
  // (independent of each other: built on host threads, kept in subdomain order)
  const int cx = md.nx_coarse / pd.nsub_x, cy = md.ny_coarse / pd.nsub_y;
  struct Sub {
    int region, i0, i1, j0, j1, di0, di1, dj0, dj1;
  };
  std::vector<Sub> subs;
  for (int region = 0; region < 2; ++region) {
    const Mesh& m = region == 0 ? L.mch : L.mph;
    const std::vector<int>& fy = region == 0 ? b.fy_c : b.fy_p;
    for (int sb = 0; sb < pd.nsub_y; ++sb)
      for (int sa = 0; sa < pd.nsub_x; ++sa) {
        int di0 = b.fx[sa * cx], di1 = b.fx[(sa + 1) * cx];
        int dj0 = fy[sb * cy], dj1 = fy[(sb + 1) * cy];
        int i0 = di0 > 0 ? std::max(di0 - pd.overlap, 0) : 0;
        int i1 = di1 < m.nx ? std::min(di1 + pd.overlap, m.nx) : m.nx;
        int j0 = dj0 > 0 ? std::max(dj0 - pd.overlap, 0) : 0;
        int j1 = dj1 < m.ny ? std::min(dj1 + pd.overlap, m.ny) : m.ny;
        subs.push_back({region, i0, i1, j0, j1, di0, di1, dj0, dj1});
      }
  }
  std::vector<Problem> probs(subs.size());
  std::vector<std::string> errs(subs.size());
  parallel_for((int)subs.size(), [&](int i) {
    const Sub& u = subs[i];
    try {
      make_problem(probs[i], u.region == 0 ? L.mch : L.mph, u.region == 0 ? PK_OSEEN : PK_DARCY, u.region, false,
                   u.i0, u.i1, u.j0, u.j1, u.di0, u.di1, u.dj0, u.dj1);
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
  make_problem(L.cfl, L.mcH, PK_OSEEN, 0, true, 0, L.mcH.nx, 0, L.mcH.ny, 0, L.mcH.nx, 0, L.mcH.ny);
  if (!finish_problem(L.cfl)) return kLongRun;
  make_problem(L.cpo, L.mpH, PK_DARCY, 1, true, 0, L.mpH.nx, 0, L.mpH.ny, 0, L.mpH.nx, 0, L.mpH.ny);
  if (!finish_problem(L.cpo)) return kLongRun;
  // Gamma partner nodes (same half-grid column on the other region's Gamma row)
  auto gam = [](Problem& P, const Mesh& self, const Mesh& other, int region) {
    P.gam_src.assign(P.nn, -1);
    const int nI = 2 * (P.i1 - P.i0) + 1;
    int Jg = region == 0 ? 0 : 2 * self.ny;
    int Jo = region == 0 ? 2 * other.ny : 0;
    for (int l = 0; l < P.nn; ++l) {
      int I = 2 * P.i0 + l % nI, J = 2 * P.j0 + l / nI;
      if (J == Jg) P.gam_src[l] = other.half_at(I, Jo);
    }
  };
  for (auto& P : L.fluid) gam(P, L.mch, L.mph, 0);
  for (auto& P : L.porous) gam(P, L.mph, L.mch, 1);
  gam(L.cfl, L.mcH, L.mpH, 0);
  gam(L.cpo, L.mpH, L.mcH, 1);
  // prolongation tables
  prolong_table(L.mcH, L.mch.node.data(), L.mch.nn, 6, L.pc2_idx, L.pc2_w);
  prolong_table(L.mcH, L.mch.node.data(), L.mch.nv, 3, L.pc1_idx, L.pc1_w);
  prolong_table(L.mpH, L.mph.node.data(), L.mph.nn, 6, L.pp2_idx, L.pp2_w);
  // glue tables
  glue_table(L.fluid, L.mch.nn, false, L.gc_ptr, L.gc_prob, L.gc_node, L.gc_w);
  glue_table(L.porous, L.mph.nn, false, L.gp_ptr, L.gp_prob, L.gp_node, L.gp_w);
  glue_table(L.fluid, L.mch.nv, true, L.gv_ptr, L.gv_prob, L.gv_vert, L.gv_w);
  for (int i = 0; i < L.mch.nn; ++i)
    if (L.gc_ptr[i + 1] == L.gc_ptr[i]) return "a conduit node is in no D_j";
  for (int i = 0; i < L.mph.nn; ++i)
    if (L.gp_ptr[i + 1] == L.gp_ptr[i]) return "a porous node is in no D_j";
  return split_ranks(L, rank, nranks);
}

// Keep this rank's local problems and their glue entries (no-op for one rank).
std::string split_ranks(Layout& L, int rank, int nranks) {
  if (nranks > 1) {
    if (rank < 0 || rank >= nranks || nranks > (int)L.fluid.size() || nranks > (int)L.porous.size())
      return "invalid rank split: nranks must not exceed the subdomains per region";
    for (int region = 0; region < 2; ++region) {
      std::vector<Problem>& list = region == 0 ? L.fluid : L.porous;
      const std::vector<int> mine = owned(list, rank, nranks);
      std::vector<int> remap(list.size(), -1);
      std::vector<Problem> kept;
      for (int i : mine) {
        remap[i] = (int)kept.size();
        kept.push_back(std::move(list[i]));
      }
      list.swap(kept);
      if (region == 0) {
        filter_glue(L.gc_ptr, L.gc_prob, L.gc_node, L.gc_w, remap);
        filter_glue(L.gv_ptr, L.gv_prob, L.gv_vert, L.gv_w, remap);
      } else {
        filter_glue(L.gp_ptr, L.gp_prob, L.gp_node, L.gp_w, remap);
      }
    }
  }
  return "";
}

// ------------------------------------------------------------------------------ reference tables
void build_ref_tables(RefTables& R) {
  // 7-point degree-5 rule on the reference triangle (Radon), closed forms in sqrt(15)
  const double s15 = std::sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
  const double w1 = (155.0 - s15) / 2400.0, w2 = (155.0 + s15) / 2400.0;
  const double P[7][2] = {{1.0 / 3.0, 1.0 / 3.0}, {a1, a1}, {1.0 - 2.0 * a1, a1}, {a1, 1.0 - 2.0 * a1},
                          {a2, a2}, {1.0 - 2.0 * a2, a2}, {a2, 1.0 - 2.0 * a2}};
  const double W[7] = {9.0 / 80.0, w1, w1, w1, w2, w2, w2};
  double N[7][6], D[7][6][2], Q[7][3];
  for (int q = 0; q < 7; ++q) {
    double x = P[q][0], y = P[q][1];
    R.qp[q][0] = x; R.qp[q][1] = y; R.qw[q] = W[q];
    double l[3] = {1 - x - y, x, y};
    const double dl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
    for (int i = 0; i < 3; ++i) {
      N[q][i] = l[i] * (2 * l[i] - 1);
      for (int r = 0; r < 2; ++r) D[q][i][r] = (4 * l[i] - 1) * dl[i][r];
    }
    const int pr[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int k = 0; k < 3; ++k) {
      int a = pr[k][0], c = pr[k][1];
      N[q][3 + k] = 4 * l[a] * l[c];
      for (int r = 0; r < 2; ++r) D[q][3 + k][r] = 4 * (l[a] * dl[c][r] + l[c] * dl[a][r]);
    }
    for (int i = 0; i < 6; ++i) R.qphi[q][i] = N[q][i];
    Q[q][0] = l[0]; Q[q][1] = l[1]; Q[q][2] = l[2];
  }
  std::fill(&R.M[0][0], &R.M[0][0] + 36, 0.0);
  std::fill(&R.S[0][0][0][0], &R.S[0][0][0][0] + 144, 0.0);
  std::fill(&R.T[0][0][0][0], &R.T[0][0][0][0] + 432, 0.0);
  std::fill(&R.U[0][0][0][0], &R.U[0][0][0][0] + 432, 0.0);
  std::fill(&R.B[0][0][0], &R.B[0][0][0] + 36, 0.0);
  for (int q = 0; q < 7; ++q)
    for (int i = 0; i < 6; ++i) {
      for (int j = 0; j < 6; ++j) {
        R.M[i][j] += W[q] * N[q][i] * N[q][j];
        for (int r = 0; r < 2; ++r)
          for (int s = 0; s < 2; ++s) R.S[i][j][r][s] += W[q] * D[q][i][r] * D[q][j][s];
        for (int k = 0; k < 6; ++k)
          for (int r = 0; r < 2; ++r) {
            R.T[k][j][i][r] += W[q] * N[q][k] * D[q][j][r] * N[q][i];
            R.U[i][j][k][r] += W[q] * N[q][i] * N[q][j] * D[q][k][r];
          }
      }
      for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 2; ++r) R.B[k][i][r] += W[q] * Q[q][k] * D[q][i][r];
    }
  // 3-point Gauss-Legendre on [0,1] and the P2 edge basis (left, right, mid)
  const double g = 0.5 * std::sqrt(3.0 / 5.0);
  const double es[3] = {0.5 - g, 0.5, 0.5 + g}, ew[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double ep[3][3], ed[3][3];
  for (int q = 0; q < 3; ++q) {
    double s = es[q];
    R.es[q] = s; R.ew[q] = ew[q];
    ep[q][0] = (1 - s) * (1 - 2 * s); ep[q][1] = s * (2 * s - 1); ep[q][2] = 4 * s * (1 - s);
    ed[q][0] = 4 * s - 3; ed[q][1] = 4 * s - 1; ed[q][2] = 4 - 8 * s;
    for (int a = 0; a < 3; ++a) R.ephi[q][a] = ep[q][a];
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      R.eM[a][c] = 0; R.eD[a][c] = 0;
      for (int q = 0; q < 3; ++q) {
        R.eM[a][c] += ew[q] * ep[q][a] * ep[q][c];
        R.eD[a][c] += ew[q] * ep[q][a] * ed[q][c];
      }
    }
}

}  // namespace tpns
