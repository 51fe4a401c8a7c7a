// Element kernels of the 3D configurations (P2/P1 tetrahedra): the local and coarse Oseen
// element matrices and right-hand sides (Alg. 3 Step 3(2), eq. uclocalFully; Step 1, eq.
// pcFully through the same residual), and the Darcy element matrices / right-hand sides
// (eqs. pFlocalFully, pflocalFully, pmlocalFully), in FP64.  The reference integrals of the
// P2/P1 basis (exact, from the 27-point rule) live in shared memory; each CTA loops over
// groups of elements (persistent grid), so the tables are read from L2 once per CTA.
#include <cuda_runtime.h>

#include "kernels.hpp"
#include "setup.hpp"

namespace tpns {
namespace {

constexpr int EPB = 4;           // elements per group
constexpr int OROWS = 34;        // 30 velocity slots + 4 pressure slots
constexpr int OTHREADS = EPB * OROWS;
constexpr int DROWS = 30;        // 3 fields x 10 rows
constexpr int DTHREADS = EPB * DROWS;
constexpr int GEO3 = 22;         // per element: 4 vertices (12), J^{-1} (9, row-major), |det J|
__device__ __constant__ int EIDX[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};

__device__ __forceinline__ void copy_tables3(RefTables3* dst, const double* src) {
  double* d = reinterpret_cast<double*>(dst);
  const int nd = (int)(sizeof(RefTables3) / sizeof(double));
  for (int i = threadIdx.x; i < nd; i += blockDim.x) d[i] = src[i];
}

struct Face {
  int gam;          // vertex opposite the face on Gamma, -1 none
  int sl[6];        // element slots of the face nodes (v0, v1, v2, m01, m02, m12)
  double det;       // 2 x area
  double J[4];      // in-plane inverse Jacobian, row-major: J[s*2 + c] = d xi_s / d x_c
  double x0[2], e1[2], e2[2];
};

// face geometry of element e from its vertex coordinates X (4 x 3)
__device__ void face_setup(Face& F, int code, const double* X) {
  F.gam = code;
  if (code < 0) return;
  int fv[3], n = 0;
  for (int v = 0; v < 4; ++v)
    if (v != code) fv[n++] = v;
  F.sl[0] = fv[0]; F.sl[1] = fv[1]; F.sl[2] = fv[2];
  F.sl[3] = 4 + EIDX[fv[0]][fv[1]];
  F.sl[4] = 4 + EIDX[fv[0]][fv[2]];
  F.sl[5] = 4 + EIDX[fv[1]][fv[2]];
  for (int c = 0; c < 2; ++c) {
    F.x0[c] = X[3 * fv[0] + c];
    F.e1[c] = X[3 * fv[1] + c] - F.x0[c];
    F.e2[c] = X[3 * fv[2] + c] - F.x0[c];
  }
  const double det = F.e1[0] * F.e2[1] - F.e2[0] * F.e1[1];
  F.det = fabs(det);
  F.J[0] = F.e2[1] / det;  F.J[1] = -F.e2[0] / det;
  F.J[2] = -F.e1[1] / det; F.J[3] = F.e1[0] / det;
}

struct ElemO {
  double X[12];
  double J[9];
  double ad;
  double w1[30], w0[30], en[30];
  double p1[4];
  double eB[34];
  int fixed[34];
  double what[30];      // what[k*3 + p] = sum_c w1[k][c] J[p][c]
  double fq[27][3];     // eta |det J| w_q f(x_q)
  Face F;
  double pF[6];
  double gN[7], gT[7][2];
  // per node pair (i, j): |det J| int d_c phi_i d_d phi_j (Sp[c][d]) and the convection
  // integral eta |det J| int (w . grad phi_j) phi_i, formed once for the three components
  double Sp[100][9];
  double c1[100];
};

}  // namespace

// ------------------------------------------------------------------------------ Oseen element
// 34 threads per element; thread r < 30 forms row r = 3 i + a (velocity node i, component a)
// of the 34 x 34 element matrix of
//   eta/dt (e, v) + 2 nu eta (D e, D v) + b_N(e, w, v) + b_N(w, e, v) + b(v, delta) - b(e, q)
//   + (eta nu alpha / sqrt(k_F)) <P_tau e, P_tau v>_Gamma
// and entry r of the right-hand side (minus the conduit residual of (w, p) with previous
// velocity w0 + e^n, forcing and Gamma data); rows 30..33 are the pressure rows -b(e, q).
// Dirichlet values of the fixed slots are moved to the right.
__global__ void __launch_bounds__(OTHREADS) oseen_elem3_kernel(AsmArgs A, int64_t e_begin, int64_t ne,
                                                               double* __restrict__ Ke, double* __restrict__ Re,
                                                               const int* skip) {
  if (skip && *skip) return;
  extern __shared__ double smem3[];
  RefTables3& R = *reinterpret_cast<RefTables3*>(smem3);
  ElemO* ES = reinterpret_cast<ElemO*>(smem3 + (sizeof(RefTables3) + 7) / 8);
  copy_tables3(&R, A.ref);
  const int le = threadIdx.x / OROWS, r = threadIdx.x % OROWS;
  const Phys& Ph = A.phys;
  const double t = *A.tnow;
  ElemO& E = ES[le];
  const int64_t ngroups = (ne + EPB - 1) / EPB;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t e = e_begin + grp * EPB + le;
    const bool valid = e < e_begin + ne;
    ProbDev P;
    if (valid) P = A.probs[A.eprob[e]];
    __syncthreads();   // the previous group is done with the shared element data
    if (valid) {
      if (r < 10) {
        const int l = A.e6[e * 10 + r];
        const int64_t ln = P.n_off + l;
        const int g = A.gnode[ln];
        const int kind = A.nkind[ln];
        for (int c = 0; c < 3; ++c) {
          E.w1[3 * r + c] = P.W1[3 * (int64_t)g + c];
          E.w0[3 * r + c] = P.W0[3 * (int64_t)g + c];
          E.en[3 * r + c] = P.EN[3 * (int64_t)l + c];
          E.fixed[3 * r + c] = A.node_dof[3 * ln + c] < 0;
        }
        double ub[3] = {0.0, 0.0, 0.0};
        if (kind == 1) {
          mms3_u(Ph, P.XY + 3 * (int64_t)g, t, ub);
          for (int c = 0; c < 3; ++c) ub[c] -= E.w1[3 * r + c];
        }
        for (int c = 0; c < 3; ++c) E.eB[3 * r + c] = ub[c];
      } else if (r < 14) {
        const int k = r - 10;
        const int lv = A.e3[e * 4 + k];
        const int l = A.vloc[P.v_off + lv];
        const int g = A.gnode[P.n_off + l];
        E.p1[k] = P.P1[g];
        E.fixed[30 + k] = A.vert_dof[P.v_off + lv] < 0;
        E.eB[30 + k] = 0.0;
      } else if (r == 14) {
        const double* gg = A.geo + e * GEO3;
        for (int q = 0; q < 12; ++q) E.X[q] = gg[q];
        for (int q = 0; q < 9; ++q) E.J[q] = gg[12 + q];
        E.ad = gg[21];
        face_setup(E.F, A.egam[e], E.X);
      }
    }
    __syncthreads();
    if (valid) {
      if (r < 27) {
        double x[3];
        for (int c = 0; c < 3; ++c)
          x[c] = E.X[c] + (E.X[3 + c] - E.X[c]) * R.qp[r][0] + (E.X[6 + c] - E.X[c]) * R.qp[r][1] +
                 (E.X[9 + c] - E.X[c]) * R.qp[r][2];
        double f[3];
        mms3_f(Ph, x, t, f);
        const double s = Ph.eta * E.ad * R.qw[r];
        for (int c = 0; c < 3; ++c) E.fq[r][c] = s * f[c];
      } else if (r == 27) {
        for (int k = 0; k < 10; ++k)
          for (int p = 0; p < 3; ++p)
            E.what[3 * k + p] = E.w1[3 * k] * E.J[3 * p] + E.w1[3 * k + 1] * E.J[3 * p + 1] +
                                E.w1[3 * k + 2] * E.J[3 * p + 2];
      } else if (r == 28 && E.F.gam >= 0) {
        for (int q = 0; q < 7; ++q) {
          const double x = E.F.x0[0] + E.F.e1[0] * R.fqp[q][0] + E.F.e2[0] * R.fqp[q][1];
          const double y = E.F.x0[1] + E.F.e1[1] * R.fqp[q][0] + E.F.e2[1] * R.fqp[q][1];
          E.gN[q] = mms3_gN(Ph, x, y, t);
          mms3_gT(Ph, x, y, t, E.gT[q]);
        }
      } else if (r == 29 && E.F.gam >= 0) {
        for (int b = 0; b < 6; ++b) {
          const int l = A.e6[e * 10 + E.F.sl[b]];
          E.pF[b] = P.GAM[A.gam_src[P.n_off + l]];
        }
      }
    }
    __syncthreads();   // what, fq, face data ready
    // the pair quantities (three pairs per thread)
    if (valid) {
      const double* J = E.J;
      const double ad = E.ad;
      for (int q = r; q < 100; q += OROWS) {
        const int i = q / 10, j = q % 10;
        double tq[3][3];
        for (int p = 0; p < 3; ++p)
          for (int d = 0; d < 3; ++d)
            tq[p][d] = R.S[i][j][p][0] * J[d] + R.S[i][j][p][1] * J[3 + d] + R.S[i][j][p][2] * J[6 + d];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d)
            E.Sp[q][3 * c + d] = ad * (J[c] * tq[0][d] + J[3 + c] * tq[1][d] + J[6 + c] * tq[2][d]);
        double c1 = 0.0;
        for (int k = 0; k < 10; ++k)
          c1 += E.what[3 * k] * R.T[k][j][i][0] + E.what[3 * k + 1] * R.T[k][j][i][1] +
                E.what[3 * k + 2] * R.T[k][j][i][2];
        E.c1[q] = ad * c1;
      }
    }
    __syncthreads();
    if (!valid) continue;
    const double eta = Ph.eta, nueta = Ph.nu * Ph.eta, eta_dt = Ph.eta / Ph.dt, ad = E.ad;
    const double* J = E.J;
    double K[34];
    double res = 0.0;
    if (r < 30) {
      const int i = r / 3, a = r % 3;
#pragma unroll
      for (int j = 0; j < 10; ++j) {
        const double* Sp = E.Sp[10 * i + j];
        double Sba[3];
        for (int b = 0; b < 3; ++b) Sba[b] = Sp[3 * b + a];
        const double lap = Sp[0] + Sp[4] + Sp[8];
        const double mij = ad * R.M[i][j];
        const double c1 = E.c1[10 * i + j];
        double u0 = 0.0, u1 = 0.0, u2 = 0.0;
        for (int k = 0; k < 10; ++k) {
          const double wk = E.w1[3 * k + a];
          u0 += wk * R.U[i][j][k][0];
          u1 += wk * R.U[i][j][k][1];
          u2 += wk * R.U[i][j][k][2];
        }
        for (int b = 0; b < 3; ++b) {
          const double visc = nueta * (Sba[b] + (a == b ? lap : 0.0));
          double v = visc + eta * ad * (J[b] * u0 + J[3 + b] * u1 + J[6 + b] * u2);
          if (a == b) v += eta_dt * mij + eta * c1;
          K[3 * j + b] = v;
          res += visc * E.w1[3 * j + b];
        }
        res += eta_dt * mij * (E.w1[3 * j + a] - E.w0[3 * j + a] - E.en[3 * j + a]) + eta * c1 * E.w1[3 * j + a];
      }
      for (int k = 0; k < 4; ++k) {
        const double v = -eta * ad * (J[a] * R.B[k][i][0] + J[3 + a] * R.B[k][i][1] + J[6 + a] * R.B[k][i][2]);
        K[30 + k] = v;
        res += v * E.p1[k];
      }
      double rhs = 0.0;
      for (int q = 0; q < 27; ++q) rhs += E.fq[q][a] * R.qphi[q][i];
      if (E.F.gam >= 0) {
        int pa = -1;
        for (int b = 0; b < 6; ++b)
          if (E.F.sl[b] == i) pa = b;
        if (pa >= 0) {
          const double kF = Ph.k[0], fd = E.F.det;
          if (a < 2) {
            const double bjs = eta * Ph.nu * Ph.alpha / sqrt(kF);
            double mb[6];
            for (int b = 0; b < 6; ++b) {
              mb[b] = bjs * fd * R.fM[pa][b];
              res += mb[b] * E.w1[3 * E.F.sl[b] + a];
            }
            // add to the row entries of the face nodes (static register indices)
#pragma unroll
            for (int j = 0; j < 10; ++j) {
              double add = 0.0;
#pragma unroll
              for (int b = 0; b < 6; ++b) add += E.F.sl[b] == j ? mb[b] : 0.0;
              if (a == 0) K[3 * j] += add;
              else K[3 * j + 1] += add;
            }
            double d = 0.0, g = 0.0;
            for (int q = 0; q < 7; ++q) {
              double gb = 0.0;
              for (int b = 0; b < 6; ++b)
                gb += E.pF[b] * (R.fdphi[q][b][0] * E.F.J[a] + R.fdphi[q][b][1] * E.F.J[2 + a]);
              d += R.fqw[q] * R.fphi[q][pa] * gb;
              g += R.fqw[q] * E.gT[q][a] * R.fphi[q][pa];
            }
            rhs += -(eta * Ph.nu * Ph.alpha * sqrt(kF) / Ph.mu) * fd * d - eta * fd * g;
          } else {
            double m = 0.0, g = 0.0;
            for (int b = 0; b < 6; ++b) m += R.fM[pa][b] * E.pF[b];
            for (int q = 0; q < 7; ++q) g += R.fqw[q] * E.gN[q] * R.fphi[q][pa];
            rhs += (eta / Ph.rho) * fd * m + eta * fd * g;
          }
        }
      }
      res = rhs - res;
    } else {
      const int k = r - 30;
#pragma unroll
      for (int j = 0; j < 10; ++j)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const double v = eta * ad * (J[b] * R.B[k][j][0] + J[3 + b] * R.B[k][j][1] + J[6 + b] * R.B[k][j][2]);
          K[3 * j + b] = v;
          res += v * E.w1[3 * j + b];
        }
      K[30] = K[31] = K[32] = K[33] = 0.0;
      res = -res;
    }
#pragma unroll
    for (int c = 0; c < 34; ++c)
      if (E.fixed[c]) res -= K[c] * E.eB[c];
    double* ko = Ke + e * (OROWS * OROWS) + r * OROWS;
#pragma unroll
    for (int c = 0; c < 34; ++c) ko[c] = K[c];
    Re[e * OROWS + r] = res;
  }
}

namespace {

struct ElemD {
  double X[12];
  double J[9];
  double ad;
  int l[10], g[10], kind[10];
  double lag[3][10];    // phiC_f/dt (p0_f + e_f) + partner exchange terms, at the nodes
  double w1[3][10];     // new coarse pressures at the nodes
  double eB[3][10];     // Dirichlet values of the correction
  double fq[27][3];     // |det J| w_q q_f(x_q)
  Face F;
  double gd[3][7];      // Gamma flux defects at the face points
  double ucn[6];        // u^n . n_c at the face nodes (partner velocities)
  double Kst[100];      // int grad phi_i . grad phi_j (reference integrals and J^{-1}, without |det J|)
};

}  // namespace

// ------------------------------------------------------------------------------ Darcy element
// 30 threads per element: thread (f, i) forms row i of A_f = (phiC_f/dt + c_f) M + (k_f/mu) K
// (written once when Ke != NULL) or entry i of the right-hand side of field f:
//   (q_f, v) - A_f p1_f + phiC_f/dt M (p0_f + e_f^n) + sum_partners c M (p0_p + e_p^n)
//   [+ <u^n . n_c, v>_Gamma for F] - <g_f, v>_Gamma, Dirichlet values moved to the right.
__global__ void __launch_bounds__(DTHREADS) darcy_elem3_kernel(AsmArgs A, int64_t e_begin, int64_t ne,
                                                               double* __restrict__ Re, double* __restrict__ Ke) {
  extern __shared__ double smem3[];
  RefTables3& R = *reinterpret_cast<RefTables3*>(smem3);
  ElemD* ES = reinterpret_cast<ElemD*>(smem3 + (sizeof(RefTables3) + 7) / 8);
  copy_tables3(&R, A.ref);
  const int le = threadIdx.x / DROWS, r = threadIdx.x % DROWS;
  const int f = r / 10, i = r % 10;
  const Phys& Ph = A.phys;
  const double t = *A.tnow;
  ElemD& E = ES[le];
  const double kf = Ph.k[1], km = Ph.k[2], mu = Ph.mu;
  const double cFf = Ph.sigma_star * kf / mu, cfm = Ph.sigma * km / mu;
  const int64_t ngroups = (ne + EPB - 1) / EPB;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t e = e_begin + grp * EPB + le;
    const bool valid = e < e_begin + ne;
    ProbDev P;
    if (valid) P = A.probs[A.eprob[e]];
    __syncthreads();
    if (valid) {
      if (r < 10) {
        const int l = A.e6[e * 10 + r];
        E.l[r] = l;
        E.g[r] = A.gnode[P.n_off + l];
        E.kind[r] = A.nkind[P.n_off + l];
      } else if (r == 10) {
        const double* gg = A.geo + e * GEO3;
        for (int q = 0; q < 12; ++q) E.X[q] = gg[q];
        for (int q = 0; q < 9; ++q) E.J[q] = gg[12 + q];
        E.ad = gg[21];
        face_setup(E.F, A.egam[e], E.X);
      }
    }
    __syncthreads();
    if (valid) {
      // the stiffness integrals, shared by the three fields
      const double* J = E.J;
      for (int q = r; q < 100; q += DROWS) {
        const int i2 = q / 10, j2 = q % 10;
        double s = 0.0;
        for (int c = 0; c < 3; ++c)
          s += R.S[i2][j2][0][0] * J[c] * J[c] + R.S[i2][j2][1][1] * J[3 + c] * J[3 + c] +
               R.S[i2][j2][2][2] * J[6 + c] * J[6 + c] + (R.S[i2][j2][0][1] + R.S[i2][j2][1][0]) * J[c] * J[3 + c] +
               (R.S[i2][j2][0][2] + R.S[i2][j2][2][0]) * J[c] * J[6 + c] +
               (R.S[i2][j2][1][2] + R.S[i2][j2][2][1]) * J[3 + c] * J[6 + c];
        E.Kst[q] = s;
      }
    }
    if (valid && !Ke) {
      if (r < 27) {
        double x[3];
        for (int c = 0; c < 3; ++c)
          x[c] = E.X[c] + (E.X[3 + c] - E.X[c]) * R.qp[r][0] + (E.X[6 + c] - E.X[c]) * R.qp[r][1] +
                 (E.X[9 + c] - E.X[c]) * R.qp[r][2];
        double q3[3];
        mms3_q3(Ph, x, t, q3);
        for (int fl = 0; fl < 3; ++fl) E.fq[r][fl] = E.ad * R.qw[r] * q3[fl];
      }
      // node values per field: thread (f, i) fills node i of field f
      {
        const int64_t gi = E.g[i];
        const int li = E.l[i];
        auto src0 = [&](int fl) { return P.W0[fl * P.fstride + gi] + P.EN[(int64_t)fl * P.nn + li]; };
        const double sC = Ph.phiC[f] / Ph.dt;
        double v = sC * src0(f);
        if (f == 0) v += cFf * src0(1);
        if (f == 1) v += cfm * src0(2) + cFf * src0(0);
        if (f == 2) v += cfm * src0(1);
        E.lag[f][i] = v;
        E.w1[f][i] = P.W1[f * P.fstride + gi];
        E.eB[f][i] = E.kind[i] == 1 ? mms3_pd(Ph, f, P.XY + 3 * gi, t) - E.w1[f][i] : 0.0;
      }
      if (E.F.gam >= 0) {
        if (r >= 27 && r < 30) {
          const int fl = r - 27;
          for (int q = 0; q < 7; ++q) {
            const double x = E.F.x0[0] + E.F.e1[0] * R.fqp[q][0] + E.F.e2[0] * R.fqp[q][1];
            const double y = E.F.x0[1] + E.F.e1[1] * R.fqp[q][0] + E.F.e2[1] * R.fqp[q][1];
            E.gd[fl][q] = mms3_gd(Ph, fl, x, y, t);
          }
        } else if (r >= 10 && r < 16) {
          const int b = r - 10;
          const int l = E.l[E.F.sl[b]];
          E.ucn[b] = -P.GAM[3 * (int64_t)A.gam_src[P.n_off + l] + 2];
        }
      }
    }
    __syncthreads();
    if (!valid) continue;
    const double ad = E.ad;
    const double cself = f == 0 ? cFf : (f == 1 ? cfm + cFf : cfm);
    const double af = Ph.phiC[f] / Ph.dt + cself, bf = Ph.k[f] / mu;
    double Arow[10];
    for (int j = 0; j < 10; ++j) Arow[j] = ad * (af * R.M[i][j] + bf * E.Kst[10 * i + j]);
    if (Ke) {
      double* ko = Ke + ((e - e_begin) * 3 + f) * 100 + i * 10;
      for (int j = 0; j < 10; ++j) ko[j] = Arow[j];
      continue;
    }
    double v = 0.0;
    for (int q = 0; q < 27; ++q) v += E.fq[q][f] * R.qphi[q][i];
    for (int j = 0; j < 10; ++j) {
      v += ad * R.M[i][j] * E.lag[f][j] - Arow[j] * E.w1[f][j];
      if (E.kind[j] > 0) v -= Arow[j] * E.eB[f][j];
    }
    if (E.F.gam >= 0) {
      int pa = -1;
      for (int b = 0; b < 6; ++b)
        if (E.F.sl[b] == i) pa = b;
      if (pa >= 0) {
        double g = 0.0, m = 0.0;
        for (int q = 0; q < 7; ++q) g += R.fqw[q] * E.gd[f][q] * R.fphi[q][pa];
        if (f == 0)
          for (int b = 0; b < 6; ++b) m += R.fM[pa][b] * E.ucn[b];
        v += E.F.det * (m - g);
      }
    }
    Re[((e - e_begin) * 3 + f) * 10 + i] = v;
  }
}

namespace {

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 132;
  }
  return n;
}

size_t smem_o() { return ((sizeof(RefTables3) + 7) / 8) * 8 + EPB * sizeof(ElemO); }
size_t smem_d() { return ((sizeof(RefTables3) + 7) / 8) * 8 + EPB * sizeof(ElemD); }

}  // namespace

cudaError_t launch_oseen_elem3(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Ke, double* Re,
                               cudaStream_t st, const int* skip) {
  if (ne <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(oseen_elem3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_o());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t groups = (ne + EPB - 1) / EPB;
  const int grid = (int)std::min<int64_t>(groups, (int64_t)2 * sm_count());
  count_launches(1);
  oseen_elem3_kernel<<<grid, OTHREADS, smem_o(), st>>>(a, e_begin, ne, Ke, Re, skip);
  return cudaGetLastError();
}

cudaError_t launch_darcy_elem3(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Re, double* Ke,
                               cudaStream_t st) {
  if (ne <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(darcy_elem3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t groups = (ne + EPB - 1) / EPB;
  const int grid = (int)std::min<int64_t>(groups, (int64_t)2 * sm_count());
  count_launches(1);
  darcy_elem3_kernel<<<grid, DTHREADS, smem_d(), st>>>(a, e_begin, ne, Re, Ke);
  return cudaGetLastError();
}

}  // namespace tpns
