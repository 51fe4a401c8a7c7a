// Band linear algebra of the local systems (Algorithm 3 Step 3): unpivoted blocked band
// LU of the Oseen saddle-point systems every step, one-time band Cholesky of the Darcy
// systems, blocked band triangular solves and FP64 CSR residuals for iterative refinement.
//
// Storage: LU band column-major, A(i, j) at band[j * ldab + ku + i - j], ldab = kl + ku + 1
// (the unpivoted LU of a band matrix stays inside the band).  Cholesky: lower band,
// L(i, j) at band[j * ldab + i - j], ldab = kl + 1.
#include <cooperative_groups.h>

#include <cmath>

#include "kernels.hpp"

namespace cg = cooperative_groups;

namespace tpns {

// ------------------------------------------------------------------------------ fill
template <typename T>
__global__ void band_zero_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                 T* __restrict__ band, int chol, const int* skip) {
  if (skip && *skip) return;
  const SysDev S = sys[list[blockIdx.y]];
  const int64_t len = (int64_t)S.n * S.ldab;
  T* B = band + S.band_off;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    B[i] = T(0);
}

template <typename T>
__global__ void band_fill_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                 const int32_t* __restrict__ rowof, const int32_t* __restrict__ colidx,
                                 const double* __restrict__ vals, T* __restrict__ band, int chol,
                                 const int* skip) {
  if (skip && *skip) return;
  const SysDev S = sys[list[blockIdx.y]];
  T* B = band + S.band_off;
  const int32_t* ro = rowof + S.nnz_off;
  const int32_t* ci = colidx + S.nnz_off;
  const double* v = vals + S.val_off;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S.nnz; k += (int64_t)gridDim.x * blockDim.x) {
    int i = ro[k], j = ci[k];
    if (chol) {
      if (i >= j) B[(int64_t)j * S.ldab + (i - j)] = (T)v[k];
    } else {
      B[(int64_t)j * S.ldab + (S.ku + i - j)] = (T)v[k];
    }
  }
}

template <typename T>
cudaError_t launch_band_fill(const SysDev* sys, const int* list, int nsys, const int32_t* rowof,
                             const int32_t* colidx, const double* vals, T* band, int chol,
                             int64_t, cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  dim3 g(64, nsys);
  band_zero_kernel<T><<<g, 256, 0, st>>>(sys, list, band, chol, skip);
  band_fill_kernel<T><<<g, 256, 0, st>>>(sys, list, rowof, colidx, vals, band, chol, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ band LU
// One thread-block cluster of LU_CLUSTER CTAs per system.  Column blocks of LU_NB columns
// are owned round robin by the CTAs of the cluster.  Step kb: every CTA forms U12 for its
// column blocks inside the band window of panel kb and applies the trailing update
// A22 -= L21 U12 to them; the owner of block kb+1 then factors panel kb+1 (no pivoting);
// one cluster barrier per step publishes the new panel.
template <typename T>
__device__ void lu_factor_panel(T* __restrict__ AB, int n, int kl, int ku, int ldab, int kb,
                                T* __restrict__ Pn, int* status) {
  constexpr int NB = LU_NB;
  const int k0 = kb * NB, kw = min(NB, n - k0);
  const int R = min(n, k0 + kw + kl) - k0;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < R * NB; idx += nt) {
    int c = idx / R, r = idx - c * R;          // r fastest: contiguous rows of one column
    int i = k0 + r, j = k0 + c;
    T v = T(0);
    if (c < kw && i - j <= kl && j - i <= ku) v = AB[(int64_t)j * ldab + (ku + i - j)];
    Pn[r * NB + c] = v;
  }
  __syncthreads();
  for (int c = 0; c < kw; ++c) {
    T piv = Pn[c * NB + c];
    if (!(piv == piv) || piv == T(0) || isinf((double)piv)) {
      if (tid == 0) atomicOr(status, 1);
      piv = T(1);
    }
    const T inv = T(1) / piv;
    for (int r = c + 1 + tid; r < R; r += nt) {
      T l = Pn[r * NB + c] * inv;
      Pn[r * NB + c] = l;
      for (int c2 = c + 1; c2 < kw; ++c2) Pn[r * NB + c2] -= l * Pn[c * NB + c2];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < R * NB; idx += nt) {
    int c = idx / R, r = idx - c * R;
    int i = k0 + r, j = k0 + c;
    if (c < kw && i - j <= kl && j - i <= ku) AB[(int64_t)j * ldab + (ku + i - j)] = Pn[r * NB + c];
  }
  __syncthreads();
}

template <typename T>
__global__ void __cluster_dims__(LU_CLUSTER, 1, 1) __launch_bounds__(256)
band_lu_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list, T* __restrict__ band,
               int* __restrict__ status, const int* skip) {
  if (skip && *skip) return;
  constexpr int NB = LU_NB, CL = LU_CLUSTER;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int sid = list[blockIdx.x / CL];
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku, ldab = S.ldab;
  T* AB = band + S.band_off;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Pn = reinterpret_cast<T*>(smem_raw);          // (NB + kl) x NB panel, row-major
  T* Ub = Pn + (size_t)(NB + kl) * NB;             // NB x NB block of U12, row-major
  const int nblk = (n + NB - 1) / NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (rank == 0 && nblk > 0) lu_factor_panel<T>(AB, n, kl, ku, ldab, 0, Pn, status + sid);
  cluster.sync();
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, kw = min(NB, n - k0);
    const int rend = min(n, k0 + kw + kl);
    const int R = rend - k0;
    const int cb_last = min(nblk - 1, (k0 + kw - 1 + ku) / NB);
    int first_mine = kb + 1;
    while (first_mine <= cb_last && first_mine % CL != rank) ++first_mine;
    if (first_mine <= cb_last) {
      // the factored panel kb (L11 unit lower, L21) into shared memory
      for (int idx = tid; idx < R * NB; idx += blockDim.x) {
        int c = idx / R, r = idx - c * R;
        int i = k0 + r, j = k0 + c;
        T v = T(0);
        if (c < kw && i - j <= kl && j - i <= ku) v = AB[(int64_t)j * ldab + (ku + i - j)];
        Pn[r * NB + c] = v;
      }
      __syncthreads();
      for (int cb = first_mine; cb <= cb_last; cb += CL) {
        const int c0 = cb * NB, cw = min(NB, n - c0);
        // A12 block (rows k0.., cols c0..), in-band entries only
        for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
          int jj = idx / NB, ii = idx - jj * NB;
          int i = k0 + ii, j = c0 + jj;
          T v = T(0);
          if (ii < kw && jj < cw && j - i <= ku && i - j <= kl) v = AB[(int64_t)j * ldab + (ku + i - j)];
          Ub[ii * NB + jj] = v;
        }
        __syncthreads();
        // U12 = L11^{-1} A12 (column per lane)
        if (warp == 0 && lane < cw) {
          for (int ii = 1; ii < kw; ++ii) {
            T acc = Ub[ii * NB + lane];
            for (int p = 0; p < ii; ++p) acc -= Pn[ii * NB + p] * Ub[p * NB + lane];
            Ub[ii * NB + lane] = acc;
          }
        }
        __syncthreads();
        for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
          int jj = idx / NB, ii = idx - jj * NB;
          int i = k0 + ii, j = c0 + jj;
          if (ii < kw && jj < cw && j - i <= ku && i - j <= kl) AB[(int64_t)j * ldab + (ku + i - j)] = Ub[ii * NB + jj];
        }
        // trailing update of rows k0+kw .. rend-1 in this column block
        for (int rb = kw + warp * 32; rb < R; rb += nwarp * 32) {
          const int r = rb + lane;
          T l[NB];
#pragma unroll
          for (int p = 0; p < NB; ++p) l[p] = (r < R) ? Pn[r * NB + p] : T(0);
          const int i = k0 + r;
          if (r < R) {
            for (int jj = 0; jj < cw; ++jj) {
              const int j = c0 + jj;
              if (i - j > kl || j - i > ku) continue;
              T* a = AB + (int64_t)j * ldab + (ku + i - j);
              T acc = *a;
#pragma unroll
              for (int p = 0; p < NB; ++p) acc -= l[p] * Ub[p * NB + jj];
              *a = acc;
            }
          }
        }
        __syncthreads();
      }
    }
    if (kb + 1 < nblk && (kb + 1) % CL == rank) lu_factor_panel<T>(AB, n, kl, ku, ldab, kb + 1, Pn, status + sid);
    cluster.sync();
  }
}

template <typename T>
cudaError_t launch_band_lu(const SysDev* sys, const int* list, int nsys, int kl_max, T* band, T*,
                           int* status, cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  size_t smem = ((size_t)(LU_NB + kl_max) * LU_NB + LU_NB * LU_NB) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(band_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  band_lu_kernel<T><<<nsys * LU_CLUSTER, 256, smem, st>>>(sys, list, band, status, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ band Cholesky
// Right-looking column Cholesky of a lower band; one CTA per system (run once per run).
template <typename T>
__global__ void __launch_bounds__(256) band_chol_kernel(const SysDev* __restrict__ sys,
                                                        const int* __restrict__ list, T* __restrict__ band,
                                                        int* __restrict__ status) {
  const int sid = list[blockIdx.x];
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ld = S.ldab;
  T* L = band + S.band_off;
  __shared__ T dsh;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      T d = L[(int64_t)j * ld];
      if (!(d > T(0)) || isinf((double)d)) {
        atomicOr(status + sid, 1);
        d = T(1);
      }
      d = sqrt(d);
      L[(int64_t)j * ld] = d;
      dsh = d;
    }
    __syncthreads();
    const int m = min(kl, n - 1 - j);
    const T inv = T(1) / dsh;
    for (int t = threadIdx.x; t < m; t += blockDim.x) L[(int64_t)j * ld + 1 + t] *= inv;
    __syncthreads();
    // L(i, k) -= L(i, j) L(k, j) for j < k <= i <= j + m
    const int pairs = m * (m + 1) / 2;
    for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
      // map t -> (k, i) with k = j+1+a, i = k+b, b in [0, m-1-a]
      int a = (int)((2 * m + 1 - sqrt((double)(2 * m + 1) * (2 * m + 1) - 8.0 * t)) / 2);
      while (a > 0 && a * (2 * m - a + 1) / 2 > t) --a;
      while ((a + 1) * (2 * m - a) / 2 <= t) ++a;
      int b = t - a * (2 * m - a + 1) / 2;
      int k = j + 1 + a, i = k + b;
      L[(int64_t)k * ld + (i - k)] -= L[(int64_t)j * ld + (i - j)] * L[(int64_t)j * ld + (k - j)];
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_band_chol(const SysDev* sys, const int* list, int nsys, T* band, int* status,
                             cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  band_chol_kernel<T><<<nsys, 256, 0, st>>>(sys, list, band, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ solves
// One CTA per system.  The right-hand side lives in shared memory in precision T; each
// block of LU_NB rows is solved by one warp against its diagonal block (staged in shared
// memory), then the rows coupled to it by the band are updated by all threads.
template <typename T>
__global__ void __launch_bounds__(256) band_solve_kernel(const SysDev* __restrict__ sys,
                                                         const int* __restrict__ list,
                                                         const int* __restrict__ chol_flag,
                                                         const T* __restrict__ band,
                                                         const double* __restrict__ rhs,
                                                         double* __restrict__ x, int accumulate,
                                                         const int* __restrict__ done, const int* skip) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.x];
  if (done && done[sid]) return;
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku, ld = S.ldab;
  const int chol = chol_flag[sid];
  const T* AB = band + S.band_off;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  T* D = v + ((n + 1) & ~1) + 2;       // NB x NB diagonal block
  constexpr int NB = LU_NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* b = rhs + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) v[i] = (T)b[i];
  __syncthreads();
  const int nblk = (n + NB - 1) / NB;
  // lower factor entry L(i, j), i >= j
  auto Lij = [&](int i, int j) -> T {
    return chol ? AB[(int64_t)j * ld + (i - j)] : AB[(int64_t)j * ld + (ku + i - j)];
  };
  // upper factor entry U(i, j), i <= j (Cholesky: L(j, i))
  auto Uij = [&](int i, int j) -> T {
    return chol ? AB[(int64_t)i * ld + (j - i)] : AB[(int64_t)j * ld + (ku + i - j)];
  };
  const int kup = chol ? kl : ku;
  // forward: L y = b
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, kw = min(NB, n - k0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      int c = idx / NB, r = idx - c * NB;
      D[r * NB + c] = (r < kw && c < kw && r >= c && r - c <= kl) ? Lij(k0 + r, k0 + c) : T(0);
    }
    __syncthreads();
    if (warp == 0) {
      T val = lane < kw ? v[k0 + lane] : T(0);
      for (int c = 0; c < kw; ++c) {
        T yc = __shfl_sync(0xffffffffu, val, c);
        if (chol && lane == c) { val = val / D[c * NB + c]; yc = val; }
        yc = __shfl_sync(0xffffffffu, val, c);
        if (lane > c) val -= D[lane * NB + c] * yc;
      }
      if (lane < kw) v[k0 + lane] = val;
    }
    __syncthreads();
    const int rend = min(n, k0 + kw + kl);
    for (int i = k0 + kw + tid; i < rend; i += blockDim.x) {
      T acc = v[i];
      const int p0 = max(k0, i - kl);
      for (int p = p0; p < k0 + kw; ++p) acc -= Lij(i, p) * v[p];
      v[i] = acc;
    }
    __syncthreads();
  }
  // backward: U x = y
  for (int kb = nblk - 1; kb >= 0; --kb) {
    const int k0 = kb * NB, kw = min(NB, n - k0);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      int c = idx / NB, r = idx - c * NB;
      D[r * NB + c] = (r < kw && c < kw && r <= c && c - r <= kup) ? Uij(k0 + r, k0 + c) : T(0);
    }
    __syncthreads();
    if (warp == 0) {
      T val = lane < kw ? v[k0 + lane] : T(0);
      for (int c = kw - 1; c >= 0; --c) {
        if (lane == c) val = val / D[c * NB + c];
        T xc = __shfl_sync(0xffffffffu, val, c);
        if (lane < c) val -= D[lane * NB + c] * xc;
      }
      if (lane < kw) v[k0 + lane] = val;
    }
    __syncthreads();
    const int rbeg = max(0, k0 - kup);
    for (int i = rbeg + tid; i < k0; i += blockDim.x) {
      T acc = v[i];
      const int p1 = min(k0 + kw, i + kup + 1);
      for (int p = k0; p < p1; ++p) acc -= Uij(i, p) * v[p];
      v[i] = acc;
    }
    __syncthreads();
  }
  double* xo = x + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) xo[i] = accumulate ? xo[i] + (double)v[i] : (double)v[i];
}

template <typename T>
cudaError_t launch_band_solve(const SysDev* sys, const int* list, const int* chol, int nsys, int n_max,
                              const T* band, const double* r, double* x, int accumulate, const int* done,
                              cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  size_t smem = ((size_t)((n_max + 1) & ~1) + 2 + LU_NB * LU_NB) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  band_solve_kernel<T><<<nsys, 256, smem, st>>>(sys, list, chol, band, r, x, accumulate, done, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ residual
// r = b - A x (FP64 CSR), relative residual and refinement control.  Stops a system when
// ||r|| <= tol ||b|| or when the residual stagnates (||r_k|| > 0.5 ||r_{k-1}||).
__global__ void __launch_bounds__(256) residual_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                       const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colidx,
                                                       const double* __restrict__ vals,
                                                       const double* __restrict__ b, const double* __restrict__ x,
                                                       double* __restrict__ r, double* __restrict__ rel,
                                                       double* __restrict__ rel_prev, int* __restrict__ done,
                                                       int* __restrict__ iters, double tol, int first,
                                                       const int* skip) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.x];
  if (!first && done[sid]) return;
  const SysDev S = sys[sid];
  const int32_t* rp = rowptr + S.rp_off;
  const int32_t* ci = colidx + S.nnz_off;
  const double* va = vals + S.val_off;
  const double* bb = b + S.x_off;
  const double* xx = x + S.x_off;
  double* rr = r + S.x_off;
  double sr = 0, sb = 0;
  for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
    double acc = bb[i];
    if (!first)
      for (int k = rp[i]; k < rp[i + 1]; ++k) acc -= va[k] * xx[ci[k]];
    rr[i] = acc;
    sr += acc * acc;
    sb += bb[i] * bb[i];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sr;
  red[1][threadIdx.x] = sb;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nb = sqrt(red[1][0]);
    double relres = nb > 0 ? sqrt(red[0][0]) / nb : 0.0;
    if (first) {
      done[sid] = (nb == 0.0) ? 1 : 0;
      iters[sid] = 0;
      rel_prev[sid] = 1.0;
      rel[sid] = nb == 0.0 ? 0.0 : 1.0;
    } else {
      iters[sid] += 1;
      double prev = rel[sid];
      rel_prev[sid] = prev;
      rel[sid] = relres;
      if (relres <= tol || relres > 0.5 * prev || !(relres == relres)) done[sid] = 1;
    }
  }
}

cudaError_t launch_residual(const SysDev* sys, const int* list, int nsys, const int32_t* rowptr,
                            const int32_t* colidx, const double* vals, const double* b, const double* x,
                            double* r, double* rel, double* rel_prev, int* done, int* iters, double tol,
                            int first, cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  residual_kernel<<<nsys, 256, 0, st>>>(sys, list, rowptr, colidx, vals, b, x, r, rel, rel_prev, done,
                                        iters, tol, first, skip);
  return cudaGetLastError();
}

#define TPNS_INST(T)                                                                                      \
  template cudaError_t launch_band_fill<T>(const SysDev*, const int*, int, const int32_t*, const int32_t*, \
                                           const double*, T*, int, int64_t, cudaStream_t, const int*);     \
  template cudaError_t launch_band_lu<T>(const SysDev*, const int*, int, int, T*, T*, int*, cudaStream_t,  \
                                         const int*);                                                      \
  template cudaError_t launch_band_chol<T>(const SysDev*, const int*, int, T*, int*, cudaStream_t);        \
  template cudaError_t launch_band_solve<T>(const SysDev*, const int*, const int*, int, int, const T*,     \
                                            const double*, double*, int, const int*, cudaStream_t,         \
                                            const int*);
TPNS_INST(float)
TPNS_INST(double)

}  // namespace tpns
