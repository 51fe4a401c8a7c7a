// Element assembly, scatter reduction, prolongation and glue kernels of the local parallel
// two-grid method (Algorithm 3, Steps 3-4), all FP64.
//
// Element integrals of the bilinear and trilinear forms of Sec. 3.1 on affine triangles
// use reference-element integrals (computed once by the degree-5 rule), so they are exact;
// forcing and interface data are integrated with the 7-point (cells) and 3-point (edges)
// rules at run time.
#include <atomic>
#include <cmath>

#include "kernels.hpp"
#include "setup.hpp"

namespace tpns {

static std::atomic<int64_t> g_launches{0};
static thread_local int64_t t_launches = 0;   // this host thread's share (graph captures)
int64_t launch_counter() { return g_launches.load(); }
int64_t thread_launch_counter() { return t_launches; }
void count_launches(int n) {
  g_launches.fetch_add(n);
  t_launches += n;
}

namespace {

struct ElemS {
  double J[4];       // Jinv row-major: J[r*2+c] = d xi_r / d x_c
  double ad;         // |det J|
  double xy[6];
  double w1[12], w0[12], en[12];
  double p1[3];
  double eB[15];
  int fixed[15];
  double what[12];   // what[k*2+r] = sum_c w1[k][c] J[r][c]
  double fq[7][2];   // eta |K| w_q f(x_q)
  int gam;
  int sl[3];         // element slots of the Gamma edge (left, right, mid)
  double pF[3];
  double L;
  double gN[3], gT[3];
  // per node pair (i, j): |det J| int d_c phi_i d_d phi_j (Sp[c][d]) and the convection
  // integral |det J| int (w . grad phi_j) phi_i, formed once for both components
  double Sp[36][4];
  double c1[36];
};

__device__ __forceinline__ void copy_tables(RefTables* dst, const double* src) {
  double* d = reinterpret_cast<double*>(dst);
  const int nd = (int)(sizeof(RefTables) / sizeof(double));
  for (int i = threadIdx.x; i < nd; i += blockDim.x) d[i] = src[i];
}

}  // namespace

// ------------------------------------------------------------------------------ Oseen element
// 16 threads per element; thread r < 15 forms row r of the 15 x 15 element matrix of
//   eta/dt (e, v) + 2 nu eta (D e, D v) + b_N(e, w, v) + b_N(w, e, v) + b(v, delta) - b(e, q)
//   + (eta nu alpha / sqrt(k_F)) <e.tau, v.tau>_Gamma
// (slots: 2*i + a for velocity node i, component a; 12 + k for vertex k) and entry r of the
// right-hand side: minus the conduit residual of (w, p) with previous velocity w0 + e^n,
// forcing and Gamma data, with Dirichlet values of the fixed slots moved to the right.
__global__ void __launch_bounds__(128) oseen_elem_kernel(AsmArgs A, int64_t e_begin, int64_t ne,
                                                         double* __restrict__ Ke, double* __restrict__ Re,
                                                         const int* skip) {
  if (skip && *skip) return;
  __shared__ RefTables R;
  __shared__ ElemS ES[8];
  copy_tables(&R, A.ref);
  const int le = threadIdx.x >> 4, r = threadIdx.x & 15;
  const int64_t e = e_begin + (int64_t)blockIdx.x * 8 + le;
  const bool valid = e < e_begin + ne;
  const Phys& Ph = A.phys;
  const double t = *A.tnow;
  ElemS& E = ES[le];
  ProbDev P;
  if (valid) P = A.probs[A.eprob[e]];
  if (valid) {
    if (r < 6) {
      const int l = A.e6[e * 6 + r];
      const int64_t ln = P.n_off + l;
      const int g = A.gnode[ln];
      const int kind = A.nkind[ln];
      for (int c = 0; c < 2; ++c) {
        E.w1[2 * r + c] = P.W1[2 * (int64_t)g + c];
        E.w0[2 * r + c] = P.W0[2 * (int64_t)g + c];
        E.en[2 * r + c] = P.EN[2 * l + c];
        E.fixed[2 * r + c] = A.node_dof[2 * ln + c] < 0;
      }
      double ub[2] = {0.0, 0.0};
      if (kind == 1) {
        mms_u(Ph, P.XY[2 * (int64_t)g], P.XY[2 * (int64_t)g + 1], t, ub);
        ub[0] -= E.w1[2 * r];
        ub[1] -= E.w1[2 * r + 1];
      }
      E.eB[2 * r] = ub[0];
      E.eB[2 * r + 1] = ub[1];
    } else if (r < 9) {
      const int k = r - 6;
      const int lv = A.e3[e * 3 + k];
      const int l = A.vloc[P.v_off + lv];
      const int g = A.gnode[P.n_off + l];
      E.p1[k] = P.P1[g];
      E.fixed[12 + k] = A.vert_dof[P.v_off + lv] < 0;
      E.eB[12 + k] = 0.0;
    } else if (r == 9) {
      const double* gg = A.geo + e * 11;
      for (int q = 0; q < 6; ++q) E.xy[q] = gg[q];
      for (int q = 0; q < 4; ++q) E.J[q] = gg[6 + q];
      E.ad = gg[10];
      const int code = A.egam[e];
      E.gam = code;
      if (code == 0) { E.sl[0] = 0; E.sl[1] = 1; E.sl[2] = 3; }
      else if (code == 1) { E.sl[0] = 2; E.sl[1] = 1; E.sl[2] = 4; }
    }
  }
  __syncthreads();
  if (valid) {
    if (r < 7) {
      const double xi = R.qp[r][0], et = R.qp[r][1];
      const double x = E.xy[0] + (E.xy[2] - E.xy[0]) * xi + (E.xy[4] - E.xy[0]) * et;
      const double y = E.xy[1] + (E.xy[3] - E.xy[1]) * xi + (E.xy[5] - E.xy[1]) * et;
      double f[2];
      mms_f(Ph, x, y, t, f);
      const double s = Ph.eta * E.ad * R.qw[r];
      E.fq[r][0] = s * f[0];
      E.fq[r][1] = s * f[1];
    } else if (r == 7) {
      for (int k = 0; k < 6; ++k)
        for (int rr = 0; rr < 2; ++rr)
          E.what[2 * k + rr] = E.w1[2 * k] * E.J[rr * 2 + 0] + E.w1[2 * k + 1] * E.J[rr * 2 + 1];
    } else if (r >= 8 && r < 11 && E.gam >= 0) {
      const int q = r - 8;
      const int el = A.e6[e * 6 + E.sl[0]], er = A.e6[e * 6 + E.sl[1]];
      const double xl = P.XY[2 * (int64_t)A.gnode[P.n_off + el]], xr = P.XY[2 * (int64_t)A.gnode[P.n_off + er]];
      const double x = xl + R.es[q] * (xr - xl);
      E.gN[q] = mms_gN(Ph, x, t);
      E.gT[q] = mms_gT(Ph, x, t);
    } else if (r == 11 && E.gam >= 0) {
      for (int b = 0; b < 3; ++b) {
        const int l = A.e6[e * 6 + E.sl[b]];
        E.pF[b] = P.GAM[A.gam_src[P.n_off + l]];
      }
      const int el = A.e6[e * 6 + E.sl[0]], er = A.e6[e * 6 + E.sl[1]];
      E.L = fabs(P.XY[2 * (int64_t)A.gnode[P.n_off + er]] - P.XY[2 * (int64_t)A.gnode[P.n_off + el]]);
    }
  }
  __syncthreads();
  // the pair quantities (36 pairs over the element's 16 threads)
  if (valid) {
    const double* J = E.J;
    const double ad = E.ad;
    for (int q = r; q < 36; q += 16) {
      const int i = q / 6, j = q % 6;
      const double s00 = R.S[i][j][0][0], s01 = R.S[i][j][0][1], s10 = R.S[i][j][1][0], s11 = R.S[i][j][1][1];
      for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d)
          E.Sp[q][2 * c + d] =
              ad * (J[0 + c] * (J[0 + d] * s00 + J[2 + d] * s01) + J[2 + c] * (J[0 + d] * s10 + J[2 + d] * s11));
      double c1 = 0.0;
      for (int k = 0; k < 6; ++k) c1 += E.what[2 * k] * R.T[k][j][i][0] + E.what[2 * k + 1] * R.T[k][j][i][1];
      E.c1[q] = ad * c1;
    }
  }
  __syncthreads();
  if (!valid || r >= 15) return;
  const double eta = Ph.eta, nueta = Ph.nu * Ph.eta, eta_dt = Ph.eta / Ph.dt, ad = E.ad;
  const double* J = E.J;
  double K[15];
  double res = 0.0;
  if (r < 12) {
    const int i = r >> 1, a = r & 1;
    for (int j = 0; j < 6; ++j) {
      const double* Spq = E.Sp[6 * i + j];
      const double Sp[2][2] = {{Spq[0], Spq[1]}, {Spq[2], Spq[3]}};
      const double mij = ad * R.M[i][j];
      const double c1 = E.c1[6 * i + j];
      double u0 = 0.0, u1 = 0.0;
      for (int k = 0; k < 6; ++k) {
        u0 += E.w1[2 * k + a] * R.U[i][j][k][0];
        u1 += E.w1[2 * k + a] * R.U[i][j][k][1];
      }
      const double lap = Sp[0][0] + Sp[1][1];
      for (int b = 0; b < 2; ++b) {
        const double visc = nueta * (Sp[b][a] + (a == b ? lap : 0.0));
        double v = visc + eta * ad * (J[0 + b] * u0 + J[2 + b] * u1);
        if (a == b) v += eta_dt * mij + eta * c1;
        K[2 * j + b] = v;
        res += visc * E.w1[2 * j + b];
      }
      res += eta_dt * mij * (E.w1[2 * j + a] - E.w0[2 * j + a] - E.en[2 * j + a]) + eta * c1 * E.w1[2 * j + a];
    }
    for (int k = 0; k < 3; ++k) {
      const double v = -eta * ad * (J[0 + a] * R.B[k][i][0] + J[2 + a] * R.B[k][i][1]);
      K[12 + k] = v;
      res += v * E.p1[k];
    }
    double rhs = 0.0;
    for (int q = 0; q < 7; ++q) rhs += E.fq[q][a] * R.qphi[q][i];
    if (E.gam >= 0) {
      int pa = -1;
      for (int b = 0; b < 3; ++b)
        if (E.sl[b] == i) pa = b;
      if (pa >= 0) {
        const double kF = Ph.k[0];
        if (a == 0) {
          const double bjs = eta * Ph.nu * Ph.alpha / sqrt(kF);
          for (int b = 0; b < 3; ++b) {
            const double m = bjs * E.L * R.eM[pa][b];
            K[2 * E.sl[b]] += m;
            res += m * E.w1[2 * E.sl[b]];
          }
          double d = 0.0, g = 0.0;
          for (int b = 0; b < 3; ++b) d += E.pF[b] * R.eD[pa][b];
          for (int q = 0; q < 3; ++q) g += R.ew[q] * E.gT[q] * R.ephi[q][pa];
          rhs += -(eta * Ph.nu * Ph.alpha * sqrt(kF) / Ph.mu) * d - eta * E.L * g;
        } else {
          double m = 0.0, g = 0.0;
          for (int b = 0; b < 3; ++b) m += R.eM[pa][b] * E.pF[b];
          for (int q = 0; q < 3; ++q) g += R.ew[q] * E.gN[q] * R.ephi[q][pa];
          rhs += (eta / Ph.rho) * E.L * m + eta * E.L * g;
        }
      }
    }
    res = rhs - res;
  } else {
    const int k = r - 12;
    for (int j = 0; j < 6; ++j)
      for (int b = 0; b < 2; ++b) {
        const double v = eta * ad * (J[0 + b] * R.B[k][j][0] + J[2 + b] * R.B[k][j][1]);
        K[2 * j + b] = v;
        res += v * E.w1[2 * j + b];
      }
    K[12] = K[13] = K[14] = 0.0;
    res = -res;
  }
  for (int c = 0; c < 15; ++c)
    if (E.fixed[c]) res -= K[c] * E.eB[c];
  double* ko = Ke + e * 225 + r * 15;
  for (int c = 0; c < 15; ++c) ko[c] = K[c];
  Re[e * 15 + r] = res;
}

cudaError_t launch_oseen_elem(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Ke, double* Re,
                              cudaStream_t st, const int* skip) {
  if (a.dim == 3) return launch_oseen_elem3(a, e_begin, ne, Ke, Re, st, skip);
  if (ne <= 0) return cudaSuccess;
  int blocks = (int)((ne + 7) / 8);
  count_launches(1);
  oseen_elem_kernel<<<blocks, 128, 0, st>>>(a, e_begin, ne, Ke, Re, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ Darcy element
// One thread per (element, field).  A_f = (phiC_f/dt + c_f) M + (k_f/mu) K.  With Ke != NULL
// the element matrices are written (run once); otherwise the right-hand side of eqs.
// pFlocalFully / pflocalFully / pmlocalFully:
//   (q_f, v) - A_f p1_f + phiC_f/dt M (p0_f + e_f^n) + sum_partners c M (p0_p + e_p^n)
//   [+ <u^n . n_c, v>_Gamma for F] - <g_f, v>_Gamma, Dirichlet values moved to the right.
__global__ void __launch_bounds__(128) darcy_elem_kernel(AsmArgs A, int64_t e_begin, int64_t ne,
                                                         double* __restrict__ Re, double* __restrict__ Ke) {
  __shared__ RefTables R;
  copy_tables(&R, A.ref);
  __syncthreads();
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ne * 3) return;
  const int64_t e = e_begin + gid / 3;
  const int f = (int)(gid % 3);
  const ProbDev P = A.probs[A.eprob[e]];
  const Phys& Ph = A.phys;
  const double t = *A.tnow;
  const double* gg = A.geo + e * 11;
  double J[4];
  for (int q = 0; q < 4; ++q) J[q] = gg[6 + q];
  const double ad = gg[10];
  const double kF = Ph.k[0], kf = Ph.k[1], km = Ph.k[2], mu = Ph.mu;
  const double cFf = Ph.sigma_star * kf / mu, cfm = Ph.sigma * km / mu;
  const double cself = f == 0 ? cFf : (f == 1 ? cfm + cFf : cfm);
  const double af = Ph.phiC[f] / Ph.dt + cself, bf = Ph.k[f] / mu;
  (void)kF;
  // grad phi_i . grad phi_j = sum_{r,s} G[r][s] d_r phi_i d_s phi_j with the metric G = J^{-1} J^{-T}
  const double G00 = J[0] * J[0] + J[1] * J[1], G11 = J[2] * J[2] + J[3] * J[3];
  const double G01 = J[0] * J[2] + J[1] * J[3];
  double Ael[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      const double s = G00 * R.S[i][j][0][0] + G01 * (R.S[i][j][0][1] + R.S[i][j][1][0]) + G11 * R.S[i][j][1][1];
      Ael[i][j] = ad * (af * R.M[i][j] + bf * s);
    }
  if (Ke) {
    double* ko = Ke + ((e - e_begin) * 3 + f) * 36;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) ko[i * 6 + j] = Ael[i][j];
    return;
  }
  int l6[6], g6[6], kind6[6];
  for (int i = 0; i < 6; ++i) {
    l6[i] = A.e6[e * 6 + i];
    g6[i] = A.gnode[P.n_off + l6[i]];
    kind6[i] = A.nkind[P.n_off + l6[i]];
  }
  const double* W1f = P.W1 + f * P.fstride;
  const double* W0f = P.W0 + f * P.fstride;
  // lagged values entering through the mass matrix
  double lag[6];
  const double sC = Ph.phiC[f] / Ph.dt;
  for (int j = 0; j < 6; ++j) {
    double v = sC * (W0f[g6[j]] + P.EN[(int64_t)f * P.nn + l6[j]]);
    if (f == 0) v += cFf * (P.W0[1 * P.fstride + g6[j]] + P.EN[(int64_t)1 * P.nn + l6[j]]);
    if (f == 1) v += cfm * (P.W0[2 * P.fstride + g6[j]] + P.EN[(int64_t)2 * P.nn + l6[j]]) +
                     cFf * (P.W0[0 * P.fstride + g6[j]] + P.EN[(int64_t)0 * P.nn + l6[j]]);
    if (f == 2) v += cfm * (P.W0[1 * P.fstride + g6[j]] + P.EN[(int64_t)1 * P.nn + l6[j]]);
    lag[j] = v;
  }
  double fq[7];
  for (int q = 0; q < 7; ++q) {
    const double xi = R.qp[q][0], et = R.qp[q][1];
    const double x = gg[0] + (gg[2] - gg[0]) * xi + (gg[4] - gg[0]) * et;
    const double y = gg[1] + (gg[3] - gg[1]) * xi + (gg[5] - gg[1]) * et;
    fq[q] = ad * R.qw[q] * mms_q(Ph, f, x, y, t);
  }
  double eB[6];
  for (int j = 0; j < 6; ++j) {
    eB[j] = 0.0;
    if (kind6[j] == 1)
      eB[j] = mms_pd(Ph, f, P.XY[2 * (int64_t)g6[j]], P.XY[2 * (int64_t)g6[j] + 1], t) - W1f[g6[j]];
  }
  // Gamma edge
  const int code = A.egam[e];
  int sl[3] = {-1, -1, -1};
  double Lg = 0.0, gq[3] = {0, 0, 0}, ucn[3] = {0, 0, 0};
  if (code >= 0) {
    if (code == 0) { sl[0] = 0; sl[1] = 1; sl[2] = 3; }
    else { sl[0] = 2; sl[1] = 1; sl[2] = 4; }
    const double xl = P.XY[2 * (int64_t)g6[sl[0]]], xr = P.XY[2 * (int64_t)g6[sl[1]]];
    Lg = fabs(xr - xl);
    for (int q = 0; q < 3; ++q) gq[q] = mms_gd(Ph, f, xl + R.es[q] * (xr - xl), t);
    if (f == 0)
      for (int b = 0; b < 3; ++b) ucn[b] = -P.GAM[2 * (int64_t)A.gam_src[P.n_off + l6[sl[b]]] + 1];
  }
  double* ro = Re + ((e - e_begin) * 3 + f) * 6;
  for (int i = 0; i < 6; ++i) {
    double v = 0.0;
    for (int q = 0; q < 7; ++q) v += fq[q] * R.qphi[q][i];
    for (int j = 0; j < 6; ++j) {
      v += ad * R.M[i][j] * lag[j] - Ael[i][j] * W1f[g6[j]];
      if (kind6[j] > 0) v -= Ael[i][j] * eB[j];
    }
    if (code >= 0) {
      int pa = -1;
      for (int b = 0; b < 3; ++b)
        if (sl[b] == i) pa = b;
      if (pa >= 0) {
        double g = 0.0, m = 0.0;
        for (int q = 0; q < 3; ++q) g += R.ew[q] * gq[q] * R.ephi[q][pa];
        for (int b = 0; b < 3; ++b) m += R.eM[pa][b] * ucn[b];
        v += Lg * (m - g);
      }
    }
    ro[i] = v;
  }
}

cudaError_t launch_darcy_elem(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Re, double* Ke,
                              cudaStream_t st) {
  if (a.dim == 3) return launch_darcy_elem3(a, e_begin, ne, Re, Ke, st);
  if (ne <= 0) return cudaSuccess;
  int blocks = (int)((ne * 3 + 127) / 128);
  count_launches(1);
  darcy_elem_kernel<<<blocks, 128, 0, st>>>(a, e_begin, ne, Re, Ke);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ scatter reduction
// Each warp reduces one 32-lane chunk of (target, source) pairs sorted by target: a
// segmented inclusive scan over runs of equal targets; the last lane of a run writes the
// sum.  Runs never straddle chunks, so every target is written exactly once, in a fixed
// order: the result is deterministic and needs no atomics.
__global__ void __launch_bounds__(256) seg_reduce_kernel(const int32_t* __restrict__ tgt,
                                                         const int32_t* __restrict__ src, int64_t nlanes,
                                                         const double* __restrict__ in, double* __restrict__ out,
                                                         const int* skip) {
  if (skip && *skip) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int t = -1;
  double v = 0.0;
  if (k < nlanes) {
    t = tgt[k];
    if (t >= 0) v = in[src[k]];
  }
  const int tprev = __shfl_up_sync(0xffffffffu, t, 1);
  const bool head = lane == 0 || tprev != t;
  // lane index of the head of this lane's run
  int hpos = head ? lane : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int o = __shfl_up_sync(0xffffffffu, hpos, d);
    if (lane >= d) hpos = max(hpos, o);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    double o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane - d >= hpos) v += o;
  }
  const int tnext = __shfl_down_sync(0xffffffffu, t, 1);
  const bool tail = lane == 31 || tnext != t;
  if (tail && t >= 0) out[t] = v;
}

cudaError_t launch_seg_reduce(const int32_t* tgt, const int32_t* src, int64_t nlanes, const double* in,
                              double* out, cudaStream_t st, const int* skip) {
  if (nlanes <= 0) return cudaSuccess;
  int blocks = (int)((nlanes + 255) / 256);
  count_launches(1);
  seg_reduce_kernel<<<blocks, 256, 0, st>>>(tgt, src, nlanes, in, out, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ state
// e^{n+1} on every local node: the solved unknown, or the Dirichlet value (I_h g - I_h I_H g
// on the global boundary, 0 on the artificial boundary); pressure 0 on the artificial boundary.
__global__ void state_kernel(AsmArgs A, const int32_t* __restrict__ nprob, const int32_t* __restrict__ nvidx,
                             int64_t n_begin, int64_t nn, const double* __restrict__ x, const int* skip) {
  if (skip && *skip) return;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nn) return;
  const int64_t ln = n_begin + gid;
  const ProbDev P = A.probs[nprob[ln]];
  const int l = (int)(ln - P.n_off);
  const int g = A.gnode[ln];
  const int kind = A.nkind[ln];
  const double t = *A.tnow;
  const Phys& Ph = A.phys;
  const int D = P.dim;
  if (P.kind == 0) {
    double ub[3] = {0.0, 0.0, 0.0};
    if (kind == 1) {
      if (D == 3) mms3_u(Ph, P.XY + 3 * (int64_t)g, t, ub);
      else mms_u(Ph, P.XY[2 * (int64_t)g], P.XY[2 * (int64_t)g + 1], t, ub);
      for (int c = 0; c < D; ++c) ub[c] -= P.W1[(int64_t)D * g + c];
    }
    for (int c = 0; c < D; ++c) {
      const int d = A.node_dof[(int64_t)D * ln + c];
      P.EOUT[(int64_t)D * l + c] = d >= 0 ? x[P.x_off + d] : ub[c];
    }
    const int v = nvidx[ln];
    if (v >= 0) {
      const int d = A.vert_dof[P.v_off + v];
      P.EOUT[(int64_t)D * P.nn + v] = d >= 0 ? x[P.x_off + d] : 0.0;
    }
  } else {
    const int d = A.node_dof[(int64_t)D * ln];
    for (int f = 0; f < 3; ++f) {
      double val;
      if (d >= 0) {
        val = x[P.x_off + (int64_t)f * P.n + d];
      } else if (kind == 1) {
        const double pd = D == 3 ? mms3_pd(Ph, f, P.XY + 3 * (int64_t)g, t)
                                 : mms_pd(Ph, f, P.XY[2 * (int64_t)g], P.XY[2 * (int64_t)g + 1], t);
        val = pd - P.W1[f * P.fstride + g];
      } else {
        val = 0.0;
      }
      P.EOUT[(int64_t)f * P.nn + l] = val;
    }
  }
}

cudaError_t launch_state(const AsmArgs& a, const int32_t* nprob, const int32_t* nvidx, int64_t n_begin,
                         int64_t nn, const double* x, cudaStream_t st, const int* skip) {
  if (nn <= 0) return cudaSuccess;
  count_launches(1);
  state_kernel<<<(int)((nn + 255) / 256), 256, 0, st>>>(a, nprob, nvidx, n_begin, nn, x, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ prolongation
// Fine nodal values of the coarse fields (fine interpolant I_h of coarse P2/P1 functions).
__global__ void prolong_kernel(int n2c, int n1c, int n2p, const int32_t* __restrict__ pc2i,
                               const double* __restrict__ pc2w, const int32_t* __restrict__ pc1i,
                               const double* __restrict__ pc1w, const int32_t* __restrict__ pp2i,
                               const double* __restrict__ pp2w, const double* __restrict__ uc_new,
                               const double* __restrict__ uc_old, const double* __restrict__ pc_new,
                               const double* __restrict__ pd_new, const double* __restrict__ pd_old,
                               int64_t nnpH, double* __restrict__ FW1, double* __restrict__ FW0,
                               double* __restrict__ FP1, double* __restrict__ FPD1,
                               double* __restrict__ FPD0, int64_t nnp, int D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nb2 = D == 3 ? 10 : 6, nb1 = D + 1;
  if (i < n2c) {
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int k = 0; k < nb2; ++k) {
      const int c = pc2i[i * nb2 + k];
      const double w = pc2w[i * nb2 + k];
      for (int d = 0; d < D; ++d) {
        a[d] += w * uc_new[(int64_t)D * c + d];
        b[d] += w * uc_old[(int64_t)D * c + d];
      }
    }
    for (int d = 0; d < D; ++d) {
      FW1[D * i + d] = a[d];
      FW0[D * i + d] = b[d];
    }
  }
  if (i < n1c) {
    double a = 0;
    for (int k = 0; k < nb1; ++k) a += pc1w[i * nb1 + k] * pc_new[pc1i[i * nb1 + k]];
    FP1[i] = a;
  }
  if (i < n2p) {
    for (int f = 0; f < 3; ++f) {
      double a = 0, b = 0;
      for (int k = 0; k < nb2; ++k) {
        const int c = pp2i[i * nb2 + k];
        const double w = pp2w[i * nb2 + k];
        a += w * pd_new[f * nnpH + c];
        b += w * pd_old[f * nnpH + c];
      }
      FPD1[f * nnp + i] = a;
      FPD0[f * nnp + i] = b;
    }
  }
}

cudaError_t launch_prolong(int n2c, int n1c, int n2p, const int32_t* pc2i, const double* pc2w,
                           const int32_t* pc1i, const double* pc1w, const int32_t* pp2i, const double* pp2w,
                           const double* uc_new, const double* uc_old, const double* pc_new,
                           const double* pd_new, const double* pd_old, int64_t nnpH, double* FW1, double* FW0,
                           double* FP1, double* FPD1, double* FPD0, int64_t nnp, cudaStream_t st, int dim) {
  int n = n2c > n2p ? n2c : n2p;
  count_launches(1);
  prolong_kernel<<<(n + 255) / 256, 256, 0, st>>>(n2c, n1c, n2p, pc2i, pc2w, pc1i, pc1w, pp2i, pp2w, uc_new,
                                                   uc_old, pc_new, pd_new, pd_old, nnpH, FW1, FW0, FP1, FPD1,
                                                   FPD0, nnp, dim);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ glue
// Step 4: fine field = I_h(coarse) + sum_j w_j e_j on the closure of D_j (w_j = 1 / number
// of closures containing the node), gathered per fine node in a fixed order.
__global__ void glue_kernel(GlueArgs G) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int D = G.dim;
  if (i < G.nnc) {
    double u[3];
    for (int d = 0; d < D; ++d) u[d] = G.add_coarse ? G.FW1[D * i + d] : 0.0;
    for (int k = G.gc_ptr[i]; k < G.gc_ptr[i + 1]; ++k) {
      const ProbDev& P = G.fluid[G.gc_prob[k]];
      const int l = G.gc_node[k];
      for (int d = 0; d < D; ++d) u[d] += G.gc_w[k] * P.EN[(int64_t)D * l + d];
    }
    for (int d = 0; d < D; ++d) G.out_u[D * i + d] = u[d];
  }
  if (i < G.nvc) {
    double p = G.add_coarse ? G.FP1[i] : 0.0;
    for (int k = G.gv_ptr[i]; k < G.gv_ptr[i + 1]; ++k) {
      const ProbDev& P = G.fluid[G.gv_prob[k]];
      p += G.gv_w[k] * P.EN[(int64_t)D * P.nn + G.gv_vert[k]];
    }
    G.out_p[i] = p;
  }
  if (i < G.nnp) {
    for (int f = 0; f < 3; ++f) {
      double v = G.add_coarse ? G.FPD1[(int64_t)f * G.nnp + i] : 0.0;
      for (int k = G.gp_ptr[i]; k < G.gp_ptr[i + 1]; ++k) {
        const ProbDev& P = G.porous[G.gp_prob[k]];
        v += G.gp_w[k] * P.EN[(int64_t)f * P.nn + G.gp_node[k]];
      }
      G.out_pd[(int64_t)f * G.nnp + i] = v;
    }
  }
}

cudaError_t launch_glue(const GlueArgs& g, cudaStream_t st) {
  int n = g.nnc > g.nnp ? g.nnc : g.nnp;
  count_launches(1);
  glue_kernel<<<(n + 255) / 256, 256, 0, st>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ coarse Newton
// u += delta, p += delta_p on the coarse conduit mesh; stop when ||delta|| <= 1e-14 ||x||.
__global__ void __launch_bounds__(256) newton_update_kernel(const ProbDev* __restrict__ prob,
                                                            const int32_t* __restrict__ gnode,
                                                            const int32_t* __restrict__ vloc, int nn, int nvl,
                                                            double* __restrict__ u, double* __restrict__ p,
                                                            int* __restrict__ done, int* __restrict__ iters) {
  if (*done) return;
  const ProbDev P = *prob;
  const double* d = P.EOUT;
  double sd = 0, sx = 0;
  const int D = P.dim;
  for (int l = threadIdx.x; l < nn; l += blockDim.x) {
    const int g = gnode[P.n_off + l];
    for (int c = 0; c < D; ++c) {
      const double v = u[(int64_t)D * g + c] + d[(int64_t)D * l + c];
      u[(int64_t)D * g + c] = v;
      sd += d[(int64_t)D * l + c] * d[(int64_t)D * l + c];
      sx += v * v;
    }
  }
  for (int v = threadIdx.x; v < nvl; v += blockDim.x) {
    const int g = gnode[P.n_off + vloc[P.v_off + v]];
    const double val = p[g] + d[(int64_t)D * nn + v];
    p[g] = val;
    sd += d[(int64_t)D * nn + v] * d[(int64_t)D * nn + v];
    sx += val * val;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sd;
  red[1][threadIdx.x] = sx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *iters += 1;
    if (sqrt(red[0][0]) <= 1e-14 * fmax(sqrt(red[1][0]), 1e-300)) *done = 1;
  }
}

cudaError_t launch_newton_update(const ProbDev* prob, const int32_t* gnode, const int32_t* vloc, int nn, int nvl,
                                 double* u, double* p, int* done, int* iters, cudaStream_t st) {
  count_launches(1);
  newton_update_kernel<<<1, 256, 0, st>>>(prob, gnode, vloc, nn, nvl, u, p, done, iters);
  return cudaGetLastError();
}

// Second-order prediction of the local iterates from the last two steps' solutions:
// x <- 2 x - x_prev once two steps are done (x unchanged before), x_prev <- the old x.
__global__ void predict_kernel(double* __restrict__ x, double* __restrict__ xprev, int64_t n,
                               const int64_t* __restrict__ step) {
  const bool extrap = *step >= 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = x[i];
    if (extrap) x[i] = 2.0 * t - xprev[i];
    xprev[i] = t;
  }
}

cudaError_t launch_predict(double* x, double* xprev, int64_t n, const int64_t* step, cudaStream_t st) {
  count_launches(1);
  predict_kernel<<<148, 256, 0, st>>>(x, xprev, n, step);
  return cudaGetLastError();
}

__global__ void set_time_kernel(double* tnow, int64_t* step, double dt, int advance) {
  if (advance) *step += 1;
  *tnow = (double)(*step + 1) * dt;
}

cudaError_t launch_set_time(double* tnow, int64_t* step, double dt, int advance, cudaStream_t st) {
  count_launches(1);
  set_time_kernel<<<1, 1, 0, st>>>(tnow, step, dt, advance);
  return cudaGetLastError();
}

}  // namespace tpns
