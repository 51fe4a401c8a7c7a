// Host-side construction of meshes, subdomains, unknown orderings, CSR patterns and
// scatter maps for the local parallel two-grid method (Algorithm 3, Steps 1-2).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "mf.hpp"
#include "tpns.h"

namespace tpns {

// Right-triangle mesh of a rectangle (Sec. 3.2 triangulation T_H or T_h of one region).
// Numbering: vertex (i, j) -> i + (nx+1) j; triangles cell by cell (x fastest), lower
// [v(i,j), v(i+1,j), v(i+1,j+1)] then upper [v(i,j), v(i+1,j+1), v(i,j+1)]; P2 nodes are
// the vertices followed by one node per edge, edges ordered by (min vid, max vid).
struct Mesh {
  int nx = 0, ny = 0;
  std::vector<double> xs, ys;
  int nv = 0, nedge = 0, nn = 0, nt = 0;
  std::vector<double> node;      // nn x 2
  std::vector<int32_t> tri;      // nt x 3
  std::vector<int32_t> tri6;     // nt x 6: v0 v1 v2 m01 m12 m20
  std::vector<int32_t> half;     // (2ny+1) x (2nx+1): half-grid (I, J) -> P2 node
  int half_at(int I, int J) const { return half[(size_t)J * (2 * nx + 1) + I]; }
  void build(const std::vector<double>& xs_, const std::vector<double>& ys_);
};

enum ProblemKind { PK_OSEEN = 0, PK_DARCY = 1 };

// One system family on a box of cells of a region mesh: a local problem on Omega_j
// (fine mesh) or the whole-region coarse problem of Step 1.
struct Problem {
  int kind = PK_OSEEN;
  int region = 0;                // 0 conduit (fluid), 1 porous
  bool coarse = false;
  bool touches_gamma = false;
  int i0 = 0, i1 = 0, j0 = 0, j1 = 0;     // cell box of Omega_j
  int di0 = 0, di1 = 0, dj0 = 0, dj1 = 0; // cell box of D_j
  int nn = 0;                    // local P2 nodes (half-grid box, I fastest)
  std::vector<int32_t> gnode;    // local node -> region mesh node
  std::vector<int8_t> nkind;     // 0 unknown, 1 global Dirichlet, 2 artificial (zero)
  std::vector<int8_t> art;       // node on the closure of the artificial boundary
  std::vector<int8_t> inD;       // node in the closure of D_j
  int nvl = 0;
  std::vector<int32_t> vloc;     // local vertex -> local node
  std::vector<int32_t> vidx;     // local node -> local vertex or -1
  int ne = 0;
  std::vector<int32_t> etri;     // element -> region mesh triangle
  std::vector<int32_t> e6, e3;   // element local nodes / local vertices
  std::vector<int8_t> egam;      // Gamma edge code of the element: -1 none, 0 = slots (0,1,3), 1 = slots (2,1,4)
  std::vector<int32_t> gam_src;  // local node -> node of the other region (same level) on Gamma, else -1
  // unknowns in band order
  int n = 0, kl = 0, ku = 0;
  std::vector<int32_t> slot_dof; // element slot -> dof (-1 if fixed): ne x S
  std::vector<int32_t> dof_node, dof_comp;   // dof -> (local node, comp) ; comp 2 = pressure
  std::vector<int32_t> node_dof; // Oseen: local node*2 + c -> dof ; Darcy: node -> dof
  std::vector<int32_t> vert_dof; // Oseen: local vertex -> dof or -1
  std::vector<int32_t> rowptr, colidx, rowof;
  // packed scatter maps: warp chunks of 32 lanes, target -1 = padding
  std::vector<int32_t> mtgt, msrc;   // element matrix entry -> CSR entry
  std::vector<int32_t> rtgt, rsrc;   // element vector entry -> unknown
  double lu_flops = 0;               // sum over columns of 2 * (#L entries) * (#U entries) + (#L)
  MFSymbolic mf;                     // multifrontal analysis (local problems)
  int slots() const { return kind == PK_OSEEN ? 15 : 6; }
};

struct Layout {
  Mesh mcH, mch, mpH, mph;       // coarse/fine conduit, coarse/fine porous
  std::vector<Problem> fluid;    // local Oseen problems
  std::vector<Problem> porous;   // local Darcy problems
  Problem cfl, cpo;              // coarse whole-region problems
  // prolongation of coarse functions to fine nodes: 6 (P2) / 3 (P1) coarse nodes + weights
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

}  // namespace tpns
