// Host-side construction of meshes, subdomains, unknown orderings, CSR patterns and
// scatter maps for the local parallel two-grid method (Algorithm 3, Steps 1-2).
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "mf.hpp"
#include "tpns.h"

namespace tpns {

// Right-triangle mesh of a rectangle (Sec. 3.2 triangulation T_H or T_h of one region).
// Numbering: vertex (i, j) -> i + (nx+1) j; triangles cell by cell (x fastest), lower
// [v(i,j), v(i+1,j), v(i+1,j+1)] then upper [v(i,j), v(i+1,j+1), v(i,j+1)]; P2 nodes are
// the vertices followed by one node per edge, edges ordered by (min vid, max vid).
//
// 3D (dim = 3): Kuhn tetrahedral mesh of a box.  Vertex (i, j, k) -> i + (nx+1)(j + (ny+1) k);
// cells x fastest, then y, then z; every cell split into the six tetrahedra
// [v000, v000 + e_a, v000 + e_a + e_b, v111] for the axis permutations (a, b, c) in
// lexicographic order; P2 nodes: vertices, then edges by (min vid, max vid); local node order
// v0..v3 then the midpoints of the edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).  Every
// point of the half grid (I, J, K) is a P2 node.
struct Mesh {
  int dim = 2;
  int nx = 0, ny = 0, nz = 0;
  std::vector<double> xs, ys, zs;
  int nv = 0, nedge = 0, nn = 0, nt = 0;
  int vpe = 3, npe = 6;          // vertices / P2 nodes per element
  std::vector<double> node;      // nn x dim
  std::vector<int32_t> tri;      // nt x vpe (triangles, or tetrahedra in 3D)
  std::vector<int32_t> tri6;     // nt x npe: 2D v0 v1 v2 m01 m12 m20; 3D see above
  std::vector<int32_t> half;     // half-grid (I, J[, K]) -> P2 node, I fastest
  int half_at(int I, int J) const { return half[(size_t)J * (2 * nx + 1) + I]; }
  int half_at3(int I, int J, int K) const {
    return half[((size_t)K * (2 * ny + 1) + J) * (2 * nx + 1) + I];
  }
  void build(const std::vector<double>& xs_, const std::vector<double>& ys_);
  void build3(const std::vector<double>& xs_, const std::vector<double>& ys_, const std::vector<double>& zs_);
};

enum ProblemKind { PK_OSEEN = 0, PK_DARCY = 1 };

// One system family on a box of cells of a region mesh: a local problem on Omega_j
// (fine mesh) or the whole-region coarse problem of Step 1.
struct Problem {
  int kind = PK_OSEEN;
  int dim = 2;
  int region = 0;                // 0 conduit (fluid), 1 porous
  bool coarse = false;
  bool touches_gamma = false;
  int i0 = 0, i1 = 0, j0 = 0, j1 = 0;     // cell box of Omega_j
  int di0 = 0, di1 = 0, dj0 = 0, dj1 = 0; // cell box of D_j
  int k0 = 0, k1 = 0, dk0 = 0, dk1 = 0;   // 3D: third axis of both boxes
  int nn = 0;                    // local P2 nodes (half-grid box, I fastest)
  std::vector<int32_t> gnode;    // local node -> region mesh node
  std::vector<int8_t> nkind;     // 0 unknown, 1 global Dirichlet, 2 artificial (zero)
  std::vector<int8_t> art;       // node on the closure of the artificial boundary
  std::vector<int8_t> inD;       // node in the closure of D_j
  int nvl = 0;
  std::vector<int32_t> vloc;     // local vertex -> local node
  std::vector<int32_t> vidx;     // local node -> local vertex or -1
  int ne = 0;
  std::vector<int32_t> etri;     // element -> region mesh element
  std::vector<int32_t> e6, e3;   // element local nodes (npe) / local vertices (vpe)
  std::vector<int8_t> egam;      // Gamma code of the element: 2D edge, -1 none, 0 = slots (0,1,3), 1 = slots (2,1,4);
                                 // 3D face, -1 none, else the local vertex opposite the face on Gamma
  std::vector<int32_t> gam_src;  // local node -> node of the other region (same level) on Gamma, else -1
  // unknowns in band order
  int n = 0, kl = 0, ku = 0;
  std::vector<int32_t> slot_dof; // element slot -> dof (-1 if fixed): ne x S
  std::vector<int32_t> dof_node, dof_comp;   // dof -> (local node, comp) ; comp 2 = pressure
  std::vector<int32_t> node_dof; // Oseen: local node*dim + c -> dof ; Darcy: node -> dof
  std::vector<int32_t> vert_dof; // Oseen: local vertex -> dof or -1
  std::vector<int32_t> rowptr, colidx, rowof;
  // packed scatter maps: warp chunks of 32 lanes, target -1 = padding
  std::vector<int32_t> mtgt, msrc;   // element matrix entry -> CSR entry
  std::vector<int32_t> rtgt, rsrc;   // element vector entry -> unknown
  double lu_flops = 0;               // sum over columns of 2 * (#L entries) * (#U entries) + (#L)
  MFSymbolic mf;                     // multifrontal analysis (local problems)
  int npe() const { return dim == 3 ? 10 : 6; }
  int vpe() const { return dim == 3 ? 4 : 3; }
  int vslots() const { return dim * npe(); }     // velocity slots of an Oseen element
  int slots() const { return kind == PK_OSEEN ? vslots() + vpe() : npe(); }
};

struct Layout {
  int dim = 2;
  Mesh mcH, mch, mpH, mph;       // coarse/fine conduit, coarse/fine porous
  std::vector<Problem> fluid;    // local Oseen problems
  std::vector<Problem> porous;   // local Darcy problems
  Problem cfl, cpo;              // coarse whole-region problems
  // prolongation of coarse functions to fine nodes: npe (P2) / vpe (P1) coarse nodes + weights
  std::vector<int32_t> pc2_idx, pc1_idx, pp2_idx;
  std::vector<double> pc2_w, pc1_w, pp2_w;
  // glue: per fine node, contributions (problem index, local node) and weight
  std::vector<int32_t> gc_ptr, gc_prob, gc_node;  // conduit P2 nodes
  std::vector<double> gc_w;
  std::vector<int32_t> gp_ptr, gp_prob, gp_node;  // porous P2 nodes
  std::vector<double> gp_w;
  // P1 glue on conduit vertices
  std::vector<int32_t> gv_ptr, gv_prob, gv_vert;
  std::vector<double> gv_w;
};

// Build everything from the ABI descriptors; returns "" on success or an error message.
// mf_leaf > 0: also run the multifrontal analysis of every local system with leaves of at
// most mf_leaf unknowns.
// rank / nranks > 1: keep only this rank's local problems (estimated per-step work, largest
// first to the least loaded rank, per region); the glue tables keep the weights of the
// whole partition but only the entries of the kept problems.
std::string build_layout(const tpns_mesh_desc& md, const tpns_partition_desc& pd, Layout& L, int mf_leaf = 0,
                         int rank = 0, int nranks = 1);
// 3D configurations (md.dim == 3): uniform Kuhn meshes, H = 1/nx_coarse, h = H/fine_per_coarse_x
std::string build_layout3(const tpns_mesh_desc& md, const tpns_partition_desc& pd, Layout& L, int mf_leaf = 0,
                          int rank = 0, int nranks = 1);

// shared by the 2D and 3D layouts
// Run task(i) for i in [0, n) on up to 16 host threads (fewer if the host has fewer or a
// thread cannot be started).  Each task must write only its own outputs and must not throw,
// so the results do not depend on the schedule.
void parallel_for(int n, const std::function<void(int)>& task);
// Build local problem i of a layout: its unknowns, CSR pattern, scatter maps and (mf_leaf >
// 0) multifrontal analysis; the error message, or "" on success.
std::string finish_local_problem(Problem& P, int mf_leaf);
bool finish_problem(Problem& P);
std::string analyse_mf(Problem& P, int leaf);
void glue_table(const std::vector<Problem>& probs, int nnodes, bool vertices, std::vector<int32_t>& ptr,
                std::vector<int32_t>& prob, std::vector<int32_t>& loc, std::vector<double>& w);
std::string split_ranks(Layout& L, int rank, int nranks);
extern const char* kLongRun;

// Reference-element integrals (computed by the degree-5 rule) and quadrature tables.
struct RefTables {
  double M[6][6];          // int phi_i phi_j
  double S[6][6][2][2];    // int d_r phi_i d_s phi_j
  double T[6][6][6][2];    // int phi_k d_r phi_j phi_i   [k][j][i][r]
  double U[6][6][6][2];    // int phi_i phi_j d_r phi_k   [i][j][k][r]
  double B[3][6][2];       // int psi_k d_r phi_i
  double qp[7][2], qw[7], qphi[7][6];
  double eM[3][3];         // int_0^1 psi_a psi_b ds (edge P2)
  double eD[3][3];         // int_0^1 psi_a psi_b' ds   [a][b]
  double es[3], ew[3], ephi[3][3];   // 3-point Gauss on [0,1]
};
void build_ref_tables(RefTables& R);

// 3D reference-element integrals (P2 / P1 tetrahedra, exact: the collapsed Gauss-Jacobi rule
// of degree 5 with 27 points) and the quadrature tables for transcendental data; the Gamma
// faces use the 7-point triangle rule with the face node order (v0, v1, v2, m01, m02, m12).
struct RefTables3 {
  double M[10][10];           // int phi_i phi_j
  double S[10][10][3][3];     // int d_r phi_i d_s phi_j
  double T[10][10][10][3];    // int phi_k d_r phi_j phi_i   [k][j][i][r]
  double U[10][10][10][3];    // int phi_i phi_j d_r phi_k   [i][j][k][r]
  double B[4][10][3];         // int psi_k d_r phi_i
  double qp[27][3], qw[27], qphi[27][10];
  double fqp[7][2], fqw[7], fphi[7][6], fdphi[7][6][2];
  double fM[6][6];            // int over the reference triangle of the face basis products
};
void build_ref_tables3(RefTables3& R);

}  // namespace tpns
