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
  count_launches(1);
  band_zero_kernel<T><<<g, 256, 0, st>>>(sys, list, band, chol, skip);
  count_launches(1);
  band_fill_kernel<T><<<g, 256, 0, st>>>(sys, list, rowof, colidx, vals, band, chol, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ band LU
// One thread-block cluster of LU_CLUSTER CTAs per system (the cluster guarantees that the
// CTAs of a system are resident together).  Column blocks of LU_NB columns are owned round
// robin by the CTAs.  At step kb every CTA waits for panel kb (L11, L21 of block kb and the
// inverses of its diagonal block), forms U12 = L11^{-1} A12 for its column blocks inside the
// band window and applies A22 -= L21 U12 to them.  The owner of block kb+1 updates that
// block first and factors panel kb+1 at once (look-ahead), then publishes it with a
// release flag; there is no barrier per step, so the CTAs run as a pipeline.
// Unpivoted: the unknown ordering makes every leading block invertible (pressures follow
// the velocities they couple to); a zero or non-finite pivot sets the status word.
constexpr int LU_THREADS = 256;
constexpr int LU_RPT = 2;                       // panel rows per thread: NB + kl <= 512
constexpr int SP = LU_NB + 1;                   // padded row stride of shared tiles

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Asynchronous global -> shared copies of one element (sizeof(T) bytes).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Inverses of the unit lower and upper triangles of a factored NB x NB diagonal block held
// in shared memory (row stride SP); written transposed (column-major) to dinv so that a
// warp reads one column per step with consecutive lanes.
template <typename T>
__device__ void diag_inverses(const T* __restrict__ D, int kw, T* __restrict__ dinv) {
  constexpr int NB = LU_NB;
  const int tid = threadIdx.x;
  if (tid < NB) {
    const int j = tid;               // column j of L11^{-1}
    T x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      T v = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int p = 0; p < i; ++p) v -= D[i * SP + p] * x[p];
      x[i] = (i < kw) ? v : T(0);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) dinv[j * NB + i] = x[i];   // dinv[p * NB + i] = Linv[i][p]
  } else if (tid < 2 * NB) {
    const int j = tid - NB;          // column j of U11^{-1}
    T x[NB];
#pragma unroll
    for (int ii = NB - 1; ii >= 0; --ii) {
      T v = (ii == j) ? T(1) : T(0);
#pragma unroll
      for (int p = ii + 1; p < NB; ++p) v -= D[ii * SP + p] * x[p];
      x[ii] = (ii < kw && j < kw) ? v / D[ii * SP + ii] : T(0);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) dinv[NB * NB + j * NB + i] = x[i];
  }
}

// Factor panel kb (columns k0..k0+kw-1, rows k0..k0+R-1) with the rows held in registers;
// the pivot row is broadcast through shared memory.  Writes the factored panel back to the
// band and the diagonal-block inverses to dinv.
template <typename T>
__device__ void lu_factor_panel_reg(T* __restrict__ AB, int n, int kl, int ku, int ldab, int kb,
                                    T* __restrict__ prow, T* __restrict__ diag, T* __restrict__ dinv,
                                    int* status) {
  constexpr int NB = LU_NB;
  const int k0 = kb * NB, kw = min(NB, n - k0);
  const int R = min(n, k0 + kw + kl) - k0;
  const int tid = threadIdx.x;
  T a[LU_RPT][NB];
#pragma unroll
  for (int q = 0; q < LU_RPT; ++q) {
    const int r = tid + q * LU_THREADS, i = k0 + r;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int j = k0 + c;
      a[q][c] = (r < R && c < kw && i - j <= kl && j - i <= ku) ? AB[(int64_t)j * ldab + (ku + i - j)] : T(0);
    }
  }
  bool bad = false;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < kw) {
      if (tid == c) {
#pragma unroll
        for (int c2 = 0; c2 < NB; ++c2) prow[c2] = a[0][c2];
      }
      __syncthreads();
      T piv = prow[c];
      if (!(piv == piv) || piv == T(0) || isinf((double)piv)) {
        bad = true;
        piv = T(1);
      }
      const T inv = T(1) / piv;
#pragma unroll
      for (int q = 0; q < LU_RPT; ++q) {
        const int r = tid + q * LU_THREADS;
        if (r > c && r < R) {
          const T l = a[q][c] * inv;
          a[q][c] = l;
#pragma unroll
          for (int c2 = c + 1; c2 < NB; ++c2) a[q][c2] -= l * prow[c2];
        }
      }
      __syncthreads();
    }
  }
  if (bad && tid == 0) atomicOr(status, 1);
#pragma unroll
  for (int q = 0; q < LU_RPT; ++q) {
    const int r = tid + q * LU_THREADS, i = k0 + r;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int j = k0 + c;
      if (r < R && c < kw && i - j <= kl && j - i <= ku) AB[(int64_t)j * ldab + (ku + i - j)] = a[q][c];
    }
  }
  if (tid < NB) {
#pragma unroll
    for (int c = 0; c < NB; ++c) diag[tid * SP + c] = a[0][c];
  }
  __syncthreads();
  diag_inverses<T>(diag, kw, dinv + (int64_t)kb * 2 * NB * NB);
}

template <typename T>
__global__ void __cluster_dims__(LU_CLUSTER, 1, 1) __launch_bounds__(LU_THREADS, 1)
band_lu_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list, T* __restrict__ band,
               T* __restrict__ dinv_all, int* __restrict__ flags_all, int flags_stride, int epoch,
               int* __restrict__ status, const int* skip) {
  if (skip && *skip) return;
  constexpr int NB = LU_NB, CL = LU_CLUSTER;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int sidx = blockIdx.x / CL;
  const int sid = list[sidx];
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku, ldab = S.ldab;
  T* AB = band + S.band_off;
  T* dinv = dinv_all + S.dinv_off;
  int* flags = flags_all + (int64_t)sid * flags_stride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Pn = reinterpret_cast<T*>(smem_raw);            // (NB + kl) x SP panel
  T* Ub = Pn + (size_t)(NB + kl) * SP;               // NB x SP block of A12 / U12
  T* Li = Ub + NB * SP;                              // NB x NB L11^{-1} (column-major)
  T* prow = Li + NB * NB;                            // NB + 1
  T* diag = prow + SP;                               // NB x SP
  __shared__ int abort_flag;
  const int nblk = (n + NB - 1) / NB;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = LU_THREADS / 32;
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  if (rank == 0 && nblk > 0) {
    lu_factor_panel_reg<T>(AB, n, kl, ku, ldab, 0, prow, diag, dinv, status + sid);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flags + 0, epoch);
    }
  }
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, kw = min(NB, n - k0);
    const int R = min(n, k0 + kw + kl) - k0;
    const int cb_last = min(nblk - 1, (k0 + kw - 1 + ku) / NB);
    int first_mine = kb + 1;
    while (first_mine <= cb_last && first_mine % CL != rank) ++first_mine;
    if (first_mine > cb_last) continue;
    // wait for panel kb (bounded; gives up with an error flag)
    if (tid == 0) {
      int it = 0;
      while (ld_acquire(flags + kb) != epoch) {
        if (++it > (1 << 22)) {
          atomicOr(status + sid, 2);
          abort_flag = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __syncthreads();
    if (abort_flag) return;
    for (int idx = tid; idx < R * NB; idx += LU_THREADS) {
      const int c = idx / R, r = idx - c * R;      // rows fastest: coalesced column reads
      const int i = k0 + r, j = k0 + c;
      if (c < kw && i - j <= kl && j - i <= ku) cp_async_elem(Pn + r * SP + c, AB + (int64_t)j * ldab + (ku + i - j));
      else Pn[r * SP + c] = T(0);
    }
    for (int idx = tid; idx < NB * NB; idx += LU_THREADS) cp_async_elem(Li + idx, dinv + (int64_t)kb * 2 * NB * NB + idx);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int cb = first_mine; cb <= cb_last; cb += CL) {
      const int c0 = cb * NB, cw = min(NB, n - c0);
      for (int idx = tid; idx < NB * NB; idx += LU_THREADS) {
        const int jj = idx / NB, ii = idx - jj * NB;
        const int i = k0 + ii, j = c0 + jj;
        if (ii < kw && jj < cw && j - i <= ku && i - j <= kl) cp_async_elem(Ub + ii * SP + jj, AB + (int64_t)j * ldab + (ku + i - j));
        else Ub[ii * SP + jj] = T(0);
      }
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      // U12 = L11^{-1} A12: four entries per thread
      T u[NB * NB / LU_THREADS];
#pragma unroll
      for (int q = 0; q < NB * NB / LU_THREADS; ++q) {
        const int idx = tid + q * LU_THREADS;
        const int jj = idx / NB, ii = idx - jj * NB;
        T acc = T(0);
#pragma unroll
        for (int p = 0; p < NB; ++p) acc += Li[p * NB + ii] * Ub[p * SP + jj];
        u[q] = acc;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NB * NB / LU_THREADS; ++q) {
        const int idx = tid + q * LU_THREADS;
        const int jj = idx / NB, ii = idx - jj * NB;
        Ub[ii * SP + jj] = u[q];
        const int i = k0 + ii, j = c0 + jj;
        if (ii < kw && jj < cw && j - i <= ku && i - j <= kl) AB[(int64_t)j * ldab + (ku + i - j)] = u[q];
      }
      __syncthreads();
      // A22 -= L21 U12 on rows kw..R-1 of this column block; lane = row
      for (int rb = kw + warp * 32; rb < R; rb += nwarp * 32) {
        const int r = rb + lane;
        const bool ok = r < R;
        T l[NB];
#pragma unroll
        for (int p = 0; p < NB; ++p) l[p] = ok ? Pn[r * SP + p] : T(0);
        const int i = k0 + r;
        if (ok) {
          // all loads of the row in flight at once, then the FMAs, then the stores
          T acc[NB];
          T* a0 = AB + (int64_t)c0 * ldab + (ku + i - c0);   // A(i, c0 + jj) = a0[jj * (ldab - 1)]
#pragma unroll
          for (int jj = 0; jj < NB; ++jj) {
            const int j = c0 + jj;
            const bool in = jj < cw && i - j <= kl && j - i <= ku;
            acc[jj] = in ? a0[(int64_t)jj * (ldab - 1)] : T(0);
          }
#pragma unroll
          for (int jj = 0; jj < NB; ++jj) {
            T t = acc[jj];
#pragma unroll
            for (int p = 0; p < NB; ++p) t -= l[p] * Ub[p * SP + jj];
            acc[jj] = t;
          }
#pragma unroll
          for (int jj = 0; jj < NB; ++jj) {
            const int j = c0 + jj;
            if (jj < cw && i - j <= kl && j - i <= ku) a0[(int64_t)jj * (ldab - 1)] = acc[jj];
          }
        }
      }
      __syncthreads();
      if (cb == kb + 1) {
        // look-ahead: block kb+1 is final up to its own panel; factor and publish it
        lu_factor_panel_reg<T>(AB, n, kl, ku, ldab, kb + 1, prow, diag, dinv, status + sid);
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release(flags + kb + 1, epoch);
        }
      }
    }
  }
}

template <typename T>
cudaError_t launch_band_lu(const SysDev* sys, const int* list, int nsys, int kl_max, T* band, T* dinv,
                           int* flags, int flags_stride, int epoch, int* status, cudaStream_t st,
                           const int* skip) {
  if (nsys == 0) return cudaSuccess;
  if (LU_NB + kl_max > LU_RPT * LU_THREADS) return cudaErrorInvalidValue;
  size_t smem = ((size_t)(LU_NB + kl_max) * SP + LU_NB * SP + LU_NB * LU_NB + SP + LU_NB * SP) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(band_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  band_lu_kernel<T><<<nsys * LU_CLUSTER, LU_THREADS, smem, st>>>(sys, list, band, dinv, flags, flags_stride, epoch,
                                                                 status, skip);
  return cudaGetLastError();
}

// Diagonal-block inverses of an already factored unit-L / U band (one CTA per system).
template <typename T>
__global__ void __launch_bounds__(LU_THREADS) band_dinv_kernel(const SysDev* __restrict__ sys,
                                                              const int* __restrict__ list, const T* __restrict__ band,
                                                              T* __restrict__ dinv_all) {
  constexpr int NB = LU_NB;
  const SysDev S = sys[list[blockIdx.x]];
  const T* AB = band + S.band_off;
  __shared__ T D[NB * SP];
  const int nblk = (S.n + NB - 1) / NB;
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, kw = min(NB, S.n - k0);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      const int c = idx / NB, r = idx - c * NB;
      const int i = k0 + r, j = k0 + c;
      D[r * SP + c] = (r < kw && c < kw && i - j <= S.kl && j - i <= S.ku) ? AB[(int64_t)j * S.ldab + (S.ku + i - j)] : T(0);
    }
    __syncthreads();
    diag_inverses<T>(D, kw, dinv_all + S.dinv_off + (int64_t)kb * 2 * NB * NB);
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_band_dinv(const SysDev* sys, const int* list, int nsys, const T* band, T* dinv, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  band_dinv_kernel<T><<<nsys, LU_THREADS, 0, st>>>(sys, list, band, dinv);
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
  count_launches(1);
  band_chol_kernel<T><<<nsys, 256, 0, st>>>(sys, list, band, status);
  return cudaGetLastError();
}


// A = L L^T = (L D^{-1}) (D L^T), D = diag(L): rewrite a lower Cholesky band (ldab_c = kl+1)
// as unit-lower / upper factors in the LU band layout (ku = kl), so that every local system
// is solved by the same triangular-solve kernel.
template <typename T>
__global__ void chol_to_lu_kernel(const SysDev* __restrict__ sys_chol, const SysDev* __restrict__ sys_lu,
                                  const int* __restrict__ list, const T* __restrict__ cband, T* __restrict__ lband) {
  const int s = list[blockIdx.y];
  const SysDev C = sys_chol[s], Lu = sys_lu[s];
  const T* Lc = cband + C.band_off;
  T* B = lband + Lu.band_off;
  const int n = C.n, kl = C.kl;
  const int64_t tot = (int64_t)n * Lu.ldab;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / Lu.ldab), off = (int)(idx % Lu.ldab);
    const int i = off - Lu.ku + j;
    T v = T(0);
    if (i >= 0 && i < n) {
      if (i > j && i - j <= kl) v = Lc[(int64_t)j * C.ldab + (i - j)] / Lc[(int64_t)j * C.ldab];
      else if (i <= j && j - i <= kl) v = Lc[(int64_t)i * C.ldab] * Lc[(int64_t)i * C.ldab + (j - i)];
    }
    B[idx] = v;
  }
}

template <typename T>
cudaError_t launch_chol_to_lu(const SysDev* sys_chol, const SysDev* sys_lu, const int* list, int nsys, const T* cband,
                              T* lband, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  chol_to_lu_kernel<T><<<dim3(64, nsys), 256, 0, st>>>(sys_chol, sys_lu, list, cband, lband);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ solves
// x (+)= U^{-1} L^{-1} r for unit-lower L and upper U in the LU band layout, one CTA per
// system.  Each block of LU_NB unknowns is finished by one warp with the stored inverse of
// its diagonal block (a GEMV), then the rows coupled to it by the band are updated by all
// threads with coalesced column reads.  The vector lives in shared memory in precision T.
template <typename T, int STAGES>
__global__ void __launch_bounds__(256) band_solve_kernel(const SysDev* __restrict__ sys,
                                                         const int* __restrict__ list,
                                                         const T* __restrict__ band, const T* __restrict__ dinv_all,
                                                         const double* __restrict__ rhs,
                                                         double* __restrict__ x, int accumulate, int kmax,
                                                         const int* __restrict__ done, const int* skip) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.x];
  if (done && done[sid]) return;
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku, ld = S.ldab;
  const T* AB = band + S.band_off;
  const T* DI = dinv_all + S.dinv_off;
  constexpr int NB = LU_NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* dib = reinterpret_cast<T*>(smem_raw);                 // STAGES x NB*NB diagonal-block inverse
  T* slab = dib + STAGES * NB * NB;                        // STAGES x NB*kmax band slab
  T* v = slab + (size_t)STAGES * NB * kmax;                // n
  __shared__ T yb[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* b = rhs + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) v[i] = (T)b[i];
  const int nblk = (n + NB - 1) / NB;
  // slab of block kb: forward  = columns k0+c, rows k0+c+1 .. k0+c+kl      (L below the diagonal)
  //                   backward = columns k0+c, rows k0+c-ku .. k0+c-1      (U above the diagonal)
  auto issue = [&](int kb, int buf, bool fwd) {
    const int k0 = kb * NB, kw = min(NB, n - k0);
    const int w = fwd ? kl : ku;
    T* sl = slab + (size_t)buf * NB * kmax;
    for (int idx = tid; idx < NB * w; idx += blockDim.x) {
      const int c = idx / w, o = idx - c * w;
      const int j = k0 + c;
      const int i = fwd ? j + 1 + o : j - ku + o;
      const int boff = fwd ? ku + 1 + o : o;
      if (c < kw && i >= 0 && i < n) cp_async_elem(sl + idx, AB + (int64_t)j * ld + boff);
      else sl[idx] = T(0);
    }
    const T* src = DI + (int64_t)kb * 2 * NB * NB + (fwd ? 0 : NB * NB);
    T* dst = dib + (size_t)buf * NB * NB;
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) cp_async_elem(dst + idx, src + idx);
    cp_async_commit();
  };
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = pass == 0;
    const int w = fwd ? kl : ku;
    issue(fwd ? 0 : nblk - 1, 0, fwd);
    for (int t = 0; t < nblk; ++t) {
      const int kb = fwd ? t : nblk - 1 - t;
      const int buf = STAGES == 2 ? (t & 1) : 0;
      if (STAGES == 2) {
        if (t + 1 < nblk) {
          issue(fwd ? kb + 1 : kb - 1, buf ^ 1, fwd);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
      } else {
        if (t > 0) issue(kb, 0, fwd);    // single buffer: fetch this block now
        cp_async_wait<0>();
      }
      __syncthreads();
      const int k0 = kb * NB, kw = min(NB, n - k0);
      const T* Dv = dib + (size_t)buf * NB * NB;
      const T* sl = slab + (size_t)buf * NB * kmax;
      if (warp == 0) {
        T acc = T(0);
#pragma unroll 8
        for (int p = 0; p < kw; ++p) acc += Dv[p * NB + lane] * v[k0 + p];
        yb[lane] = lane < kw ? acc : T(0);
      }
      __syncthreads();
      if (tid < kw) v[k0 + tid] = yb[tid];
      if (fwd) {
        const int rend = min(n, k0 + kw + kl);
        for (int i = k0 + 1 + tid; i < rend; i += blockDim.x) {
          if (i < k0 + kw) continue;
          T acc = v[i];
          // L(i, k0 + c) = sl[c * w + (i - k0 - c - 1)], valid for 0 <= i - k0 - c - 1 < kl
#pragma unroll 8
          for (int c = 0; c < kw; ++c) {
            const int o = i - k0 - c - 1;
            if (o >= 0 && o < kl) acc -= sl[c * w + o] * yb[c];
          }
          v[i] = acc;
        }
      } else {
        const int rbeg = max(0, k0 - ku);
        for (int i = rbeg + tid; i < k0; i += blockDim.x) {
          T acc = v[i];
          // U(i, k0 + c) = sl[c * w + (i - k0 - c + ku)], valid for 0 <= i - k0 - c + ku < ku
#pragma unroll 8
          for (int c = 0; c < kw; ++c) {
            const int o = i - k0 - c + ku;
            if (o >= 0 && o < ku) acc -= sl[c * w + o] * yb[c];
          }
          v[i] = acc;
        }
      }
      __syncthreads();
    }
  }
  double* xo = x + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) xo[i] = accumulate ? xo[i] + (double)v[i] : (double)v[i];
}

template <typename T>
cudaError_t launch_band_solve(const SysDev* sys, const int* list, int nsys, int n_max, int kmax, const T* band,
                              const T* dinv, const double* r, double* x, int accumulate, const int* done,
                              cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t need2 = ((size_t)2 * LU_NB * LU_NB + (size_t)2 * LU_NB * kmax + n_max + 4) * sizeof(T);
  const size_t need1 = ((size_t)LU_NB * LU_NB + (size_t)LU_NB * kmax + n_max + 4) * sizeof(T);
  count_launches(1);
  if (need2 + 1024 <= (size_t)smem_max) {
    cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need2);
    if (e != cudaSuccess) return e;
    band_solve_kernel<T, 2><<<nsys, 256, need2, st>>>(sys, list, band, dinv, r, x, accumulate, kmax, done, skip);
  } else {
    if (need1 + 1024 > (size_t)smem_max) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need1);
    if (e != cudaSuccess) return e;
    band_solve_kernel<T, 1><<<nsys, 256, need1, st>>>(sys, list, band, dinv, r, x, accumulate, kmax, done, skip);
  }
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
  count_launches(1);
  residual_kernel<<<nsys, 256, 0, st>>>(sys, list, rowptr, colidx, vals, b, x, r, rel, rel_prev, done,
                                        iters, tol, first, skip);
  return cudaGetLastError();
}

#define TPNS_INST(T)                                                                                      \
  template cudaError_t launch_band_fill<T>(const SysDev*, const int*, int, const int32_t*, const int32_t*, \
                                           const double*, T*, int, int64_t, cudaStream_t, const int*);     \
  template cudaError_t launch_band_lu<T>(const SysDev*, const int*, int, int, T*, T*, int*, int, int, int*,\
                                         cudaStream_t, const int*);                                        \
  template cudaError_t launch_band_dinv<T>(const SysDev*, const int*, int, const T*, T*, cudaStream_t);    \
  template cudaError_t launch_band_chol<T>(const SysDev*, const int*, int, T*, int*, cudaStream_t);        \
  template cudaError_t launch_chol_to_lu<T>(const SysDev*, const SysDev*, const int*, int, const T*, T*,   \
                                            cudaStream_t);                                                 \
  template cudaError_t launch_band_solve<T>(const SysDev*, const int*, int, int, int, const T*, const T*,  \
                                            const double*, double*, int, const int*, cudaStream_t,         \
                                            const int*);
TPNS_INST(float)
TPNS_INST(double)

}  // namespace tpns
