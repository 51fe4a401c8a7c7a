// Symbolic analysis of the multifrontal LU (see mf.hpp): nested dissection of the
// half-grid box of a local problem, the elimination tree, the update set of every front,
// the maps that assemble a front from the CSR values and from its children's Schur
// complements (extend-add), and the algorithmic flop count.  Pure host code.
#include <algorithm>
#include <functional>
#include <numeric>

#include "mf.hpp"

namespace tpns {

namespace {

struct Node {
  std::vector<int32_t> own;
  int nchild = 0, child[2] = {-1, -1};
};

}  // namespace

std::string mf_analyse(int n, int dim, const int32_t* coord, const int8_t* pressure, const int32_t* rowptr,
                       const int32_t* colidx, int leaf_max, MFSymbolic& out) {
  out = MFSymbolic();
  if (n <= 0 || dim < 1 || dim > 3 || leaf_max < 1) return "mf_analyse: invalid arguments";
  std::vector<Node> nodes;
  std::vector<int32_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  int lo0[3] = {0, 0, 0}, hi0[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    lo0[d] = coord[d];
    hi0[d] = coord[d];
    for (int i = 0; i < n; ++i) {
      lo0[d] = std::min(lo0[d], coord[(size_t)i * dim + d]);
      hi0[d] = std::max(hi0[d], coord[(size_t)i * dim + d]);
    }
  }
  // velocities before pressures, then by coordinates (last axis slowest), then by id
  auto own_order = [&](std::vector<int32_t>& v) {
    std::sort(v.begin(), v.end(), [&](int32_t a, int32_t b) {
      if (pressure[a] != pressure[b]) return pressure[a] < pressure[b];
      for (int d = dim - 1; d >= 0; --d) {
        int ca = coord[(size_t)a * dim + d], cb = coord[(size_t)b * dim + d];
        if (ca != cb) return ca < cb;
      }
      return a < b;
    });
  };
  // recursive bisection at vertex planes; returns the node index (postorder)
  std::function<int(std::vector<int32_t>&, const int*, const int*)> dissect =
      [&](std::vector<int32_t>& ids, const int* lo, const int* hi) -> int {
    int axis = -1, ext = 0;
    if ((int)ids.size() > leaf_max)
      for (int d = 0; d < dim; ++d)
        if (hi[d] - lo[d] >= 4 && hi[d] - lo[d] > ext) {
          ext = hi[d] - lo[d];
          axis = d;
        }
    Node node;
    if (axis >= 0) {
      int s = (lo[axis] + hi[axis]) / 2;
      if (s % 2) s += (s + 1 <= hi[axis] - 1) ? 1 : -1;
      std::vector<int32_t> left, right, sep;
      for (int32_t u : ids) {
        int c = coord[(size_t)u * dim + axis];
        (c < s ? left : c > s ? right : sep).push_back(u);
      }
      int lo2[3] = {lo[0], lo[1], lo[2]}, hi2[3] = {hi[0], hi[1], hi[2]};
      hi2[axis] = s - 1;
      if (!left.empty()) node.child[node.nchild++] = dissect(left, lo, hi2);
      hi2[axis] = hi[axis];
      lo2[axis] = s + 1;
      if (!right.empty()) node.child[node.nchild++] = dissect(right, lo2, hi);
      node.own.swap(sep);
      if (node.own.empty() && node.nchild == 1) return node.child[0];   // nothing on the plane
    } else {
      node.own = ids;
    }
    own_order(node.own);
    nodes.push_back(std::move(node));
    return (int)nodes.size() - 1;
  };
  dissect(all, lo0, hi0);
  const int nf = (int)nodes.size();
  // elimination positions (postorder: children before parents)
  std::vector<int32_t> pos(n, -1), front_of(n, -1), first(nf), last(nf);
  out.order.clear();
  for (int t = 0; t < nf; ++t) {
    first[t] = (int)out.order.size();
    for (int c = 0; c < nodes[t].nchild; ++c) first[t] = std::min(first[t], first[nodes[t].child[c]]);
    for (int32_t u : nodes[t].own) {
      pos[u] = (int32_t)out.order.size();
      front_of[u] = t;
      out.order.push_back(u);
    }
    last[t] = (int)out.order.size() - 1;
  }
  if ((int)out.order.size() != n) return "mf_analyse: dissection lost unknowns";
  // update sets bottom-up
  out.fronts.assign(nf, MFFront());
  std::vector<int32_t> mark(n, -1), idx(n, -1);
  for (int t = 0; t < nf; ++t) {
    MFFront& F = out.fronts[t];
    const Node& N = nodes[t];
    F.p = (int)N.own.size();
    F.nchild = N.nchild;
    std::vector<int32_t> upd;
    auto consider = [&](int32_t v) {
      if (pos[v] > last[t] && mark[v] != t) {
        mark[v] = t;
        upd.push_back(v);
      }
    };
    for (int c = 0; c < N.nchild; ++c) {
      const MFFront& C = out.fronts[N.child[c]];
      F.child[c] = N.child[c];
      out.fronts[N.child[c]].parent = t;
      for (int i = C.p; i < C.m; ++i) consider(C.rows[i]);
    }
    for (int32_t u : N.own)
      for (int k = rowptr[u]; k < rowptr[u + 1]; ++k) {
        int32_t v = colidx[k];
        if (pos[v] < first[t]) return "mf_analyse: a separator does not separate";
        consider(v);
      }
    std::sort(upd.begin(), upd.end(), [&](int32_t a, int32_t b) { return pos[a] < pos[b]; });
    F.rows = N.own;
    F.rows.insert(F.rows.end(), upd.begin(), upd.end());
    F.m = (int)F.rows.size();
    F.level = 0;
    for (int c = 0; c < N.nchild; ++c) F.level = std::max(F.level, out.fronts[N.child[c]].level + 1);
    out.nlevels = std::max(out.nlevels, F.level + 1);
  }
  // relmaps, originals, column maps of children
  for (int t = 0; t < nf; ++t) {
    MFFront& F = out.fronts[t];
    for (int i = 0; i < F.m; ++i) idx[F.rows[i]] = i;
    for (int c = 0; c < F.nchild; ++c) {
      MFFront& C = out.fronts[F.child[c]];
      C.relmap.resize(C.m - C.p);
      for (int i = C.p; i < C.m; ++i) {
        int32_t j = idx[C.rows[i]];
        if (j < 0) return "mf_analyse: a child's update set is not in its parent";
        C.relmap[i - C.p] = j;
      }
    }
    F.col_child.assign((size_t)F.m * 2, -1);
    for (int c = 0; c < F.nchild; ++c) {
      const MFFront& C = out.fronts[F.child[c]];
      for (int jc = 0; jc < C.m - C.p; ++jc) F.col_child[(size_t)C.relmap[jc] * 2 + c] = jc;
    }
    // an entry (u, v) belongs to the front that eliminates the earlier of u and v
    std::vector<std::pair<int32_t, std::pair<int32_t, int32_t>>> ent;   // (col, (row, k))
    for (int a = 0; a < F.p; ++a) {
      const int32_t w = F.rows[a];
      for (int k = rowptr[w]; k < rowptr[w + 1]; ++k) {
        const int32_t v = colidx[k];
        if (pos[v] < pos[w]) continue;
        if (idx[v] < 0) return "mf_analyse: an entry lies outside its front";
        ent.push_back({idx[v], {a, k}});
        if (v == w) continue;
        const int32_t* b = colidx + rowptr[v];
        const int32_t* e = colidx + rowptr[v + 1];
        const int32_t* f = std::lower_bound(b, e, w);
        if (f == e || *f != w) return "mf_analyse: pattern is not structurally symmetric";
        ent.push_back({a, {idx[v], (int32_t)(f - colidx)}});
      }
    }
    std::sort(ent.begin(), ent.end());
    F.col_ptr.assign(F.m + 1, 0);
    F.orig_k.resize(ent.size());
    F.orig_i.resize(ent.size());
    for (size_t q = 0; q < ent.size(); ++q) {
      F.col_ptr[ent[q].first + 1] += 1;
      F.orig_i[q] = ent[q].second.first;
      F.orig_k[q] = ent[q].second.second;
    }
    for (int j = 0; j < F.m; ++j) F.col_ptr[j + 1] += F.col_ptr[j];
    for (int i = 0; i < F.m; ++i) idx[F.rows[i]] = -1;
    double fl = 0;
    for (int k = 0; k < F.p; ++k) {
      const double r = F.m - 1 - k;
      fl += r + 2.0 * r * r;
    }
    out.flops += fl;
    out.factor_entries += (double)F.p * F.p + 2.0 * F.p * (F.m - F.p);
  }
  return "";
}

}  // namespace tpns
