// Device-side descriptors and the manufactured data of the two-grid method.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tpns {

// A problem family on one box: a local problem on Omega_j or a coarse whole-region
// problem (Algorithm 3 Steps 1 and 3).  Offsets index the concatenated arrays of the
// context; pointers give the sources of the coarse state and the local correction.
struct ProbDev {
  int kind;          // 0 Oseen, 1 Darcy
  int coarse;        // 1: coarse problem of Step 1
  int dim;           // 2 or 3: velocity components per node and coordinates per node
  int ne, nn, nvl, n;
  int64_t e_off;     // elements: geometry, e6, e3, egam
  int64_t n_off;     // local nodes: gnode, nkind, gam_src, node_dof (Oseen: 2 per node)
  int64_t v_off;     // local vertices: vloc, vert_dof
  int64_t x_off;     // unknown vectors (Darcy: 3 consecutive blocks of n)
  const double* W1;  // Oseen: velocity about which the problem is linearised (dim/node);
                     // Darcy: new coarse pressures (3 fields, stride `fstride`)
  const double* W0;  // Oseen: previous coarse velocity; Darcy: previous coarse pressures
  const double* P1;  // Oseen: coarse pressure at vertices (unused for Darcy)
  const double* GAM; // Oseen: porous p_F^n at Gamma partner nodes; Darcy: conduit velocity
                     // u^n (dim/node) at Gamma partner nodes
  const double* EN;  // local correction e^n read by the element kernels;
                     // Oseen: dim*nn velocity then nvl pressure; Darcy: 3 blocks of nn
  double* EOUT;      // where the new correction e^{n+1} is written (same layout; equal to
                     // EN for local problems, so the state is updated in place)
  const double* XY;  // node coordinates of the region mesh (dim/node)
  int64_t fstride;   // field stride of Darcy sources W1 / W0
};

// Linear system descriptor (one Oseen system, or one field of a Darcy problem).
struct SysDev {
  int n, kl, ku, ldab;
  int64_t band_off;  // band storage (column-major band, ldab per column)
  int64_t rp_off;    // CSR row pointer (n+1 entries)
  int64_t nnz_off;   // CSR column index / row index (pattern shared by the Darcy fields)
  int64_t nnz;       // CSR entries
  int64_t val_off;   // CSR values
  int64_t x_off;     // b, x, r vectors
  int64_t dinv_off;  // inverses of the diagonal blocks of L and U (2 * nblk * 32 * 32)
  int64_t lslab_off; // L below the diagonal, per 32-column block: [c][i - j - 1], 32 * kl per block
  int64_t uslab_off; // U above the diagonal, per 32-column block: [c][i - j + ku], 32 * ku per block
};

struct Phys {
  double nu, eta, rho, mu, alpha, sigma, sigma_star;
  double phiC[3], k[3];
  double dt;
  int mms;
};

// ---------------------------------------------------------------- manufactured data
// mms 1: u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)) e^-t, p = cos(pi x) cos(pi y) e^-t,
//        p_F, p_f, p_m = 3, 2, 1 times cos(pi x) cos(pi y) e^-t.
// mms 3: u = (x^2, -2xy), p = x + y, p_F, p_f, p_m = 3, 2, 1 times (x^2 + y^2).
// The forcing, Gamma defects and boundary data below are derived by hand from the strong
// form of Sec. 2 (see the oracle for an independent symbolic derivation).
__device__ __forceinline__ void mms_u(const Phys& P, double x, double y, double t, double* u) {
  if (P.mms == 1) {
    double sx, cx, sy, cy;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    double E = exp(-t);
    u[0] = sx * cy * E;
    u[1] = -cx * sy * E;
  } else if (P.mms == 3) {
    u[0] = x * x;
    u[1] = -2.0 * x * y;
  } else {
    u[0] = 0.0;
    u[1] = 0.0;
  }
}

__device__ __forceinline__ double mms_p(const Phys& P, double x, double y, double t) {
  if (P.mms == 1) return cospi(x) * cospi(y) * exp(-t);
  if (P.mms == 3) return x + y;
  return 0.0;
}

__device__ __forceinline__ double mms_pd(const Phys& P, int f, double x, double y, double t) {
  const double a = 3.0 - f;   // F: 3, f: 2, m: 1
  if (P.mms == 1) return a * cospi(x) * cospi(y) * exp(-t);
  if (P.mms == 3) return a * (x * x + y * y);
  return 0.0;
}

// conduit forcing f = du/dt - div T(u, p) + (u.grad)u
__device__ __forceinline__ void mms_f(const Phys& P, double x, double y, double t, double* f) {
  if (P.mms == 1) {
    const double pi = 3.141592653589793;
    double sx, cx, sy, cy;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    double E = exp(-t);
    f[0] = sx * cy * E * (-1.0 + 2.0 * P.nu * pi * pi - pi) + pi * sx * cx * E * E;
    f[1] = cx * sy * E * (1.0 - 2.0 * P.nu * pi * pi - pi) + pi * sy * cy * E * E;
  } else if (P.mms == 3) {
    f[0] = 1.0 - 2.0 * P.nu + 2.0 * x * x * x;
    f[1] = 1.0 + 2.0 * x * x * y;
  } else {
    f[0] = 0.0;
    f[1] = 0.0;
  }
}

// Darcy sources q_F, q_f, q_m of eqs. (2.1)-(2.3)
__device__ __forceinline__ double mms_q(const Phys& P, int fld, double x, double y, double t) {
  const double kF = P.k[0], kf = P.k[1], km = P.k[2], mu = P.mu;
  const double cFf = P.sigma_star * kf / mu, cfm = P.sigma * km / mu;
  if (P.mms == 1) {
    const double pi2 = 9.869604401089358;
    double C = cospi(x) * cospi(y) * exp(-t);
    if (fld == 0) return C * (-3.0 * P.phiC[0] + 6.0 * pi2 * kF / mu + cFf);
    if (fld == 1) return C * (-2.0 * P.phiC[1] + 4.0 * pi2 * kf / mu - cFf + cfm);
    return C * (-P.phiC[2] + 2.0 * pi2 * km / mu - cfm);
  }
  if (P.mms == 3) {
    double r2 = x * x + y * y;
    if (fld == 0) return -12.0 * kF / mu + cFf * r2;
    if (fld == 1) return -8.0 * kf / mu + (cfm - cFf) * r2;
    return -4.0 * km / mu - cfm * r2;
  }
  return 0.0;
}

// Interface defects on Gamma (y = 1, n_c = (0,-1), tau = (1,0)):
// g_N = -n_c.T n_c - p_F/rho,  g_T = -tau.T n_c - (alpha nu/sqrt(k_F)) tau.(u + k_F/mu grad p_F)
__device__ __forceinline__ double mms_gN(const Phys& P, double x, double t) {
  if (P.mms == 1) {
    const double pi = 3.141592653589793;
    double cx = cospi(x), E = exp(-t);
    return -(2.0 * P.nu * pi + 1.0) * cx * E + 3.0 * cx * E / P.rho;
  }
  if (P.mms == 3) return 4.0 * P.nu * x + x + 1.0 - 3.0 * (x * x + 1.0) / P.rho;
  return 0.0;
}

__device__ __forceinline__ double mms_gT(const Phys& P, double x, double t) {
  const double kF = P.k[0];
  if (P.mms == 1) {
    const double pi = 3.141592653589793;
    return P.alpha * P.nu / sqrt(kF) * sinpi(x) * exp(-t) * (1.0 - 3.0 * pi * kF / P.mu);
  }
  if (P.mms == 3) return -2.0 * P.nu - P.alpha * P.nu / sqrt(kF) * (x * x + 6.0 * x * kF / P.mu);
  return 0.0;
}

// Darcy flux defects g_F = u.n_c - k_F/mu dp_F/dy, g_f = -k_f/mu dp_f/dy, g_m = -k_m/mu dp_m/dy
__device__ __forceinline__ double mms_gd(const Phys& P, int fld, double x, double t) {
  if (P.mms == 3) {
    if (fld == 0) return 2.0 * x - 6.0 * P.k[0] / P.mu;
    if (fld == 1) return -4.0 * P.k[1] / P.mu;
    return -2.0 * P.k[2] / P.mu;
  }
  return 0.0;   // mms 1: all three vanish on y = 1
}

// ---------------------------------------------------------------- 3D manufactured data
// Gamma is z = 1, n_c = (0,0,-1), n_p = (0,0,1), P_tau v = (v_x, v_y, 0).
// mms 2: u = (sx cy cz, cx sy cz, -2 cx cy sz) e^-t (sx = sin(pi x), cx = cos(pi x), ...),
//        p = cx cy cz e^-t, p_F, p_f, p_m = 3, 2, 1 times cx cy cz e^-t (div u = 0).
// mms 4: u = (x^2, y^2, -2 (x + y) z), p = x + y + z, p_F, p_f, p_m = 3, 2, 1 times
//        (x^2 + y^2 + z^2).
// Forcing, sources and Gamma defects below are derived by hand from the strong form of
// Sec. 2 (the oracle derives them independently, symbolically).
__device__ __forceinline__ void mms3_u(const Phys& P, const double* X, double t, double* u) {
  const double x = X[0], y = X[1], z = X[2];
  if (P.mms == 2) {
    double sx, cx, sy, cy, sz, cz;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    sincospi(z, &sz, &cz);
    const double E = exp(-t);
    u[0] = sx * cy * cz * E;
    u[1] = cx * sy * cz * E;
    u[2] = -2.0 * cx * cy * sz * E;
  } else if (P.mms == 4) {
    u[0] = x * x;
    u[1] = y * y;
    u[2] = -2.0 * (x + y) * z;
  } else {
    u[0] = u[1] = u[2] = 0.0;
  }
}

__device__ __forceinline__ double mms3_pd(const Phys& P, int f, const double* X, double t) {
  const double a = 3.0 - f;
  if (P.mms == 2) return a * cospi(X[0]) * cospi(X[1]) * cospi(X[2]) * exp(-t);
  if (P.mms == 4) return a * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  return 0.0;
}

// conduit forcing f = du/dt - div T(u, p) + (u.grad)u
__device__ __forceinline__ void mms3_f(const Phys& P, const double* X, double t, double* f) {
  const double x = X[0], y = X[1], z = X[2];
  if (P.mms == 2) {
    const double pi = 3.141592653589793;
    double sx, cx, sy, cy, sz, cz;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    sincospi(z, &sz, &cz);
    const double E = exp(-t), E2 = E * E;
    const double a = 3.0 * P.nu * pi * pi - 1.0;   // -du/dt - nu lap u = (3 nu pi^2 - 1) u
    f[0] = sx * cy * cz * E * (a - pi) + pi * E2 * sx * cx * (cy * cy * cz * cz - sy * sy * cz * cz + 2.0 * cy * cy * sz * sz);
    f[1] = cx * sy * cz * E * (a - pi) + pi * E2 * sy * cy * (cx * cx * cz * cz - sx * sx * cz * cz + 2.0 * cx * cx * sz * sz);
    f[2] = cx * cy * sz * E * (-2.0 * a - pi) +
           2.0 * pi * E2 * sz * cz * (sx * sx * cy * cy + cx * cx * sy * sy + 2.0 * cx * cx * cy * cy);
  } else if (P.mms == 4) {
    f[0] = 1.0 - 2.0 * P.nu + 2.0 * x * x * x;
    f[1] = 1.0 - 2.0 * P.nu + 2.0 * y * y * y;
    f[2] = 1.0 - 2.0 * z * (x * x + y * y) + 4.0 * z * (x + y) * (x + y);
  } else {
    f[0] = f[1] = f[2] = 0.0;
  }
}

// Darcy sources q_F, q_f, q_m
__device__ __forceinline__ double mms3_q(const Phys& P, int fld, const double* X, double t) {
  const double kf = P.k[1], km = P.k[2], mu = P.mu;
  const double cFf = P.sigma_star * kf / mu, cfm = P.sigma * km / mu;
  if (P.mms == 2) {
    const double pi2 = 9.869604401089358;
    const double C = cospi(X[0]) * cospi(X[1]) * cospi(X[2]) * exp(-t);
    if (fld == 0) return C * (-3.0 * P.phiC[0] + 9.0 * pi2 * P.k[0] / mu + cFf);
    if (fld == 1) return C * (-2.0 * P.phiC[1] + 6.0 * pi2 * kf / mu - cFf + cfm);
    return C * (-P.phiC[2] + 3.0 * pi2 * km / mu - cfm);
  }
  if (P.mms == 4) {
    const double r2 = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    if (fld == 0) return -18.0 * P.k[0] / mu + cFf * r2;
    if (fld == 1) return -12.0 * kf / mu + (cfm - cFf) * r2;
    return -6.0 * km / mu - cfm * r2;
  }
  return 0.0;
}

// the three sources at one point (the trigonometric base is formed once)
__device__ __forceinline__ void mms3_q3(const Phys& P, const double* X, double t, double* q) {
  if (P.mms == 2) {
    const double kf = P.k[1], km = P.k[2], mu = P.mu;
    const double cFf = P.sigma_star * kf / mu, cfm = P.sigma * km / mu;
    const double pi2 = 9.869604401089358;
    const double C = cospi(X[0]) * cospi(X[1]) * cospi(X[2]) * exp(-t);
    q[0] = C * (-3.0 * P.phiC[0] + 9.0 * pi2 * P.k[0] / mu + cFf);
    q[1] = C * (-2.0 * P.phiC[1] + 6.0 * pi2 * kf / mu - cFf + cfm);
    q[2] = C * (-P.phiC[2] + 3.0 * pi2 * km / mu - cfm);
    return;
  }
  for (int f = 0; f < 3; ++f) q[f] = mms3_q(P, f, X, t);
}

// g_N = -n_c.T n_c - p_F/rho on z = 1
__device__ __forceinline__ double mms3_gN(const Phys& P, double x, double y, double t) {
  if (P.mms == 2) {
    const double pi = 3.141592653589793;
    const double c = cospi(x) * cospi(y) * exp(-t);
    return -(4.0 * pi * P.nu + 1.0) * c + 3.0 * c / P.rho;
  }
  if (P.mms == 4) return 4.0 * P.nu * (x + y) + x + y + 1.0 - 3.0 * (x * x + y * y + 1.0) / P.rho;
  return 0.0;
}

// g_T = -P_tau(T n_c) - (alpha nu / sqrt(k_F)) P_tau(u + k_F/mu grad p_F) on z = 1 (x, y)
__device__ __forceinline__ void mms3_gT(const Phys& P, double x, double y, double t, double* g) {
  const double kF = P.k[0], c = P.alpha * P.nu / sqrt(kF);
  if (P.mms == 2) {
    const double pi = 3.141592653589793;
    double sx, cx, sy, cy;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    const double s = c * exp(-t) * (1.0 - 3.0 * pi * kF / P.mu);
    g[0] = s * sx * cy;
    g[1] = s * cx * sy;
  } else if (P.mms == 4) {
    g[0] = -2.0 * P.nu - c * (x * x + 6.0 * x * kF / P.mu);
    g[1] = -2.0 * P.nu - c * (y * y + 6.0 * y * kF / P.mu);
  } else {
    g[0] = g[1] = 0.0;
  }
}

// g_F = u.n_c - k_F/mu dp_F/dz, g_f = -k_f/mu dp_f/dz, g_m = -k_m/mu dp_m/dz on z = 1
__device__ __forceinline__ double mms3_gd(const Phys& P, int fld, double x, double y, double t) {
  (void)t;
  if (P.mms == 4) {
    if (fld == 0) return 2.0 * (x + y) - 6.0 * P.k[0] / P.mu;
    if (fld == 1) return -4.0 * P.k[1] / P.mu;
    return -2.0 * P.k[2] / P.mu;
  }
  return 0.0;   // mms 2: all three vanish on z = 1
}

}  // namespace tpns
