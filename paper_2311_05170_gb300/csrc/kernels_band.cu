// Band linear algebra of the local systems (Algorithm 3 Step 3): unpivoted blocked band
// LU of the Oseen saddle-point systems every step, one-time band Cholesky of the Darcy
// systems, blocked band triangular solves and FP64 CSR residuals for iterative refinement.
//
// Storage: LU band column-major, A(i, j) at band[j * ldab + ku + i - j], ldab = kl + ku + 1
// (the unpivoted LU of a band matrix stays inside the band).  Cholesky: lower band,
// L(i, j) at band[j * ldab + i - j], ldab = kl + 1.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
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
// One thread-block cluster per system (8 CTAs, or 16 for very wide bands whose trailing
// updates outweigh the chain; the cluster keeps the CTAs of a system resident together).  CTA 0 produces every panel: it keeps the current factored
// panel (L11, L21) in shared memory, forms U12 of the next column block, applies
// A22 -= L21 U12 to that block while loading it into registers, factors it there (no
// pivoting) and publishes it with a release flag.  The other CTAs own the other column blocks
// round robin and apply every published panel to them, publishing per-block progress
// counters that CTA 0 waits for.  Thus the chain of panels never waits for a barrier or a
// global reload, and the bulk updates run beside it.
// Unpivoted: the unknown ordering makes every leading block invertible (pressures follow
// the velocities they couple to); a zero or non-finite pivot sets bit 0 of the status word,
// a wait that gives up sets bit 1.
// Besides the working band, the final factors are written to per-block slabs
// (L: [c][i - j - 1], U: [c][i - j + ku]) that the triangular solves stream with TMA.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// threads per LU CTA: one panel row per thread (NB + kl <= threads); 768 for FP32 and 512
// for FP64 (85 / 128 registers per thread), so that the single critical CTA has enough warps
// to hide the latency of its dependent phases
template <typename T>
__host__ __device__ constexpr int lu_threads() { return sizeof(T) == 4 ? 768 : 512; }
constexpr int SP = LU_NB + 1;                   // padded row stride of shared tiles
constexpr int WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool wait_eq(const int* p, int v) {
  for (int it = 0; ld_acquire(p) != v; ++it) {
    if (it > WAIT_LIMIT) return false;
    __nanosleep(64);
  }
  return true;
}
// progress counters hold (epoch << 12) | count
__device__ __forceinline__ int cnt_word(int epoch, int c) { return ((epoch & 0x7FFFF) << 12) | c; }
__device__ __forceinline__ bool wait_cnt(const int* p, int epoch, int need) {
  for (int it = 0;; ++it) {
    const int v = ld_acquire(p);
    if ((v >> 12) == (epoch & 0x7FFFF) && (v & 4095) >= need) return true;
    if (it > WAIT_LIMIT) return false;
    __nanosleep(64);
  }
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

// a pivot is unusable if it is zero, NaN or infinite (tested in its own precision)
__device__ __forceinline__ bool bad_pivot(float v) { return !(fabsf(v) > 0.0f) || !(fabsf(v) < INFINITY); }
__device__ __forceinline__ bool bad_pivot(double v) { return !(fabs(v) > 0.0) || !(fabs(v) < (double)INFINITY); }

__device__ __forceinline__ int64_t lsl_idx(int i, int j, int kl) {
  return (int64_t)(j >> 5) * 32 * kl + (int64_t)(j & 31) * kl + (i - j - 1);
}
__device__ __forceinline__ int64_t usl_idx(int i, int j, int ku) {
  return (int64_t)(j >> 5) * 32 * ku + (int64_t)(j & 31) * ku + (i - j + ku);
}

// Column j of the inverse of the upper triangle of a factored NB x NB diagonal block D (row
// stride SP), written to dinvU[j * NB + i].
template <typename T>
__device__ __forceinline__ void diag_upper_column(const T* __restrict__ D, int kw, int j, T* __restrict__ dinvU) {
  constexpr int NB = LU_NB;
  T x[NB];
#pragma unroll
  for (int ii = NB - 1; ii >= 0; --ii) {
    T v = (ii == j) ? T(1) : T(0);
#pragma unroll
    for (int p = ii + 1; p < NB; ++p) v -= D[ii * SP + p] * x[p];
    x[ii] = (ii < kw && j < kw) ? v / D[ii * SP + ii] : T(0);
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) dinvU[j * NB + i] = x[i];
}

// Inverses of the unit lower and upper triangles of a factored NB x NB diagonal block held
// in shared memory (row stride SP); written transposed (column-major) to dinv so that a
// warp reads one column per step with consecutive lanes.  Threads 0..63.
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
    diag_upper_column<T>(D, kw, tid - NB, dinv + NB * NB);   // column j of U11^{-1}
  }
}

// Pivot rows are broadcast through shared memory in rows of PR elements (16-byte aligned);
// element NB holds the reciprocal of the pivot.
constexpr int PR = LU_NB + 4;

// a[c2] -= l * pr[c2] for C < c2 < NB, reading pr with 16-byte vector loads
template <int C, typename T>
__device__ __forceinline__ void axpy_tail(T (&a)[LU_NB], T l, const T* __restrict__ pr) {
  constexpr int NB = LU_NB;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int g = (C + 1) / 4; g < NB / 4; ++g) {
      const float4 v = reinterpret_cast<const float4*>(pr)[g];
      if (4 * g + 0 > C) a[4 * g + 0] -= l * v.x;
      if (4 * g + 1 > C) a[4 * g + 1] -= l * v.y;
      if (4 * g + 2 > C) a[4 * g + 2] -= l * v.z;
      if (4 * g + 3 > C) a[4 * g + 3] -= l * v.w;
    }
  } else {
#pragma unroll
    for (int g = (C + 1) / 2; g < NB / 2; ++g) {
      const double2 v = reinterpret_cast<const double2*>(pr)[g];
      if (2 * g + 0 > C) a[2 * g + 0] -= l * v.x;
      if (2 * g + 1 > C) a[2 * g + 1] -= l * v.y;
    }
  }
}

// store a row of NB values and the reciprocal of its pivot as a broadcast pivot row
template <typename T>
__device__ __forceinline__ void put_pivot_row(T* __restrict__ pn, const T (&a)[LU_NB], T rcp) {
  constexpr int NB = LU_NB;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int g = 0; g < NB / 4; ++g)
      reinterpret_cast<float4*>(pn)[g] = make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
  } else {
#pragma unroll
    for (int g = 0; g < NB / 2; ++g) reinterpret_cast<double2*>(pn)[g] = make_double2(a[2 * g], a[2 * g + 1]);
  }
  pn[NB] = rcp;
}

// Column C of the factorisation of the diagonal block by warp 0, lane r holding row r: the
// pivot and the tail of pivot row C are broadcast by warp shuffles, the rows below take their
// multiplier and update their tails.
template <int C, typename T>
__device__ __forceinline__ void diag_columns(T (&a)[LU_NB], int lane, int kw, bool& bad) {
  if constexpr (C < LU_NB) {
    if (C < kw) {
      T piv = __shfl_sync(0xffffffffu, a[C], C);
      if (bad_pivot(piv)) {
        bad = true;
        piv = T(1);
      }
      const T rcp = T(1) / piv;
      const T l = a[C] * rcp;
      if (lane > C) a[C] = l;
#pragma unroll
      for (int c2 = C + 1; c2 < LU_NB; ++c2) {
        const T u = __shfl_sync(0xffffffffu, a[c2], C);
        if (lane > C) a[c2] -= l * u;
      }
      diag_columns<C + 1>(a, lane, kw, bad);
    }
  }
}

// A row below the diagonal block, against the stored pivot rows (row C of Ud: U(C, .) and
// the reciprocal of the pivot at NB), column by column with no synchronisation.
template <int C, typename T>
__device__ __forceinline__ void sub_columns(T (&a)[LU_NB], int kw, const T* __restrict__ Ud) {
  if constexpr (C < LU_NB) {
    if (C < kw) {
      const T* pr = Ud + C * PR;
      const T l = a[C] * pr[LU_NB];
      a[C] = l;
      axpy_tail<C>(a, l, pr);
      sub_columns<C + 1>(a, kw, Ud);
    }
  }
}

// Factor the panel whose rows are held in registers (row r = threadIdx.x relative to k0,
// columns k0..k0+kw-1).  Warp 0 factors the diagonal block (warp shuffles, no block
// barrier) and stores its rows, each with the reciprocal of its pivot, as the pivot rows Ud
// (NB x PR); after one barrier every other row eliminates against them on its own.  Every
// multiplier and update is the operation a right-looking elimination of the panel performs,
// in the same order.  The factored rows go to shared memory only: the L part of every row into the
// skewed buffer Lsk (NB x kl, column c at c * kl, row r at r - c - 1: the layout of the
// block's L slab, so that one bulk copy stores it, and conflict-free for lanes along rows),
// rows 0..NB-1 (the diagonal block) into Dt (row stride SP); those rows also write their U
// part to the U slab and the diagonal block into the band (for the inverses of its
// triangles).  Rows past the matrix hold zeros and fill their slots of Lsk.
template <typename T>
__device__ void factor_rows(T (&a)[LU_NB], int k0, int kw, int R, int kl, int ku, int ldab, T* __restrict__ AB,
                            T* __restrict__ US, T* __restrict__ Dt, T* __restrict__ Lsk, T* __restrict__ Ud,
                            int* status) {
  constexpr int NB = LU_NB;
  const int tid = threadIdx.x;
  const int r = tid, i = k0 + r;
  bool bad = false;
  if (tid < NB) {
    diag_columns<0>(a, tid, kw, bad);
    // this lane's pivot (the same value, hence the same reciprocal, as in its column step)
    T piv = T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c == tid) piv = a[c];
    if (bad_pivot(piv)) piv = T(1);
    put_pivot_row(Ud + tid * PR, a, T(1) / piv);
  }
  __syncthreads();
  if (r >= NB && r < R) sub_columns<0>(a, kw, Ud);
  if (bad) atomicOr(status, 1);
  if (r < NB + kl) {
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int o = r - c - 1;
      if (o >= 0 && o < kl) Lsk[c * kl + o] = a[c];
    }
  }
  if (r < NB && r < R) {
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int j = k0 + c;
      Dt[r * SP + c] = a[c];
      if (c < kw && i - j <= kl && j - i <= ku) {
        AB[(int64_t)j * ldab + (ku + i - j)] = a[c];
        if (i < j) US[usl_idx(i, j, ku)] = a[c];
      }
    }
  }
}

// Bulk copy of the skewed L buffer to the block's L slab (one thread; after a barrier that
// follows the buffer's writes).  tma_store_wait must run before the slab is published.
template <typename T>
__device__ __forceinline__ void tma_store_lslab(T* __restrict__ dst, const T* __restrict__ Lsk, int kl) {
  if (kl <= 0) return;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const unsigned src = smem_u32(Lsk);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"((unsigned)(LU_NB * kl * sizeof(T))) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Factor the panel held in shared memory Pn (row stride SP, rows 0..R-1 relative to k0,
// columns k0..k0+kw-1), for panels taller than the CTA.  Warp 0 takes rows 0..NB-1 into
// registers and factors the diagonal block as factor_rows does, leaving the pivot rows with
// their reciprocals in Ud (NB x PR); after one barrier every thread takes its rows tid + NB,
// tid + NB + THREADS, ... from Pn, eliminates them against Ud and puts them back.  Same
// operations in the same order as factor_rows, so both give the same factors.  Writes the
// slabs and the factored diagonal block into the band.
template <typename T>
__device__ void factor_panel_smem(int k0, int kw, int R, int kl, int ku, int ldab, T* __restrict__ AB,
                                  T* __restrict__ LS, T* __restrict__ US, T* __restrict__ Pn, T* __restrict__ Ud,
                                  int* status) {
  constexpr int NB = LU_NB;
  constexpr int THREADS = lu_threads<T>();
  const int tid = threadIdx.x;
  bool bad = false;
  if (tid < NB) {
    T a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = Pn[tid * SP + c];
    diag_columns<0>(a, tid, kw, bad);
    T piv = T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c == tid) piv = a[c];
    if (bad_pivot(piv)) piv = T(1);
    put_pivot_row(Ud + tid * PR, a, T(1) / piv);
#pragma unroll
    for (int c = 0; c < NB; ++c) Pn[tid * SP + c] = a[c];
  }
  if (bad) atomicOr(status, 1);
  __syncthreads();
  for (int r = NB + tid; r < R; r += THREADS) {
    T a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = Pn[r * SP + c];
    sub_columns<0>(a, kw, Ud);
#pragma unroll
    for (int c = 0; c < NB; ++c) Pn[r * SP + c] = a[c];
  }
  __syncthreads();
  for (int r = tid; r < R; r += THREADS) {
    const int i = k0 + r;
#pragma unroll 4
    for (int c = 0; c < kw; ++c) {
      const int j = k0 + c;
      if (i - j <= kl && j - i <= ku) {
        const T v = Pn[r * SP + c];
        if (r < NB) AB[(int64_t)j * ldab + (ku + i - j)] = v;
        if (i > j) LS[lsl_idx(i, j, kl)] = v;
        else if (i < j) US[usl_idx(i, j, ku)] = v;
      }
    }
  }
}

// U12 = L11^{-1} A12 for one column block: A12 (rows k0.., columns c0..) is loaded into Ub
// (row stride SP) with lanes along rows (coalesced band reads) and multiplied by the inverse
// Li (column-major, column stride ls) with lanes along columns, so that every shared-memory
// access is conflict-free: Li is read by broadcast, Ub and Uv along rows.  The result goes to
// the unpadded copy Uv used for broadcast reads, back into Ub, and from there, lanes along
// rows again, to the U slab.
template <typename T>
__device__ void form_u12(const T* __restrict__ Li, int ls, T* __restrict__ Ub, T* __restrict__ Uv,
                         const T* __restrict__ AB, T* __restrict__ US, int k0, int kw, int c0, int cw, int kl, int ku,
                         int ldab) {
  constexpr int NB = LU_NB;
  constexpr int THREADS = lu_threads<T>();
  constexpr int PER = (NB * NB + THREADS - 1) / THREADS;
  const int tid = threadIdx.x;
  T v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + q * THREADS;
    const int jj = idx / NB, ii = idx - jj * NB;          // lanes along rows
    const int i = k0 + ii, j = c0 + jj;
    v[q] = (idx < NB * NB && ii < kw && jj < cw && j - i <= ku && i - j <= kl)
               ? __ldcg(AB + (int64_t)j * ldab + (ku + i - j)) : T(0);
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + q * THREADS;
    const int jj = idx / NB, ii = idx - jj * NB;
    if (idx < NB * NB) Ub[ii * SP + jj] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + q * THREADS;
    const int ii = idx / NB, jj = idx - ii * NB;          // lanes along columns
    T acc = T(0);
    if (idx < NB * NB) {
#pragma unroll
      for (int p = 0; p < NB; ++p) acc += Li[p * ls + ii] * Ub[p * SP + jj];
    }
    v[q] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + q * THREADS;
    const int ii = idx / NB, jj = idx - ii * NB;
    if (idx < NB * NB) {
      Uv[ii * NB + jj] = v[q];
      Ub[ii * SP + jj] = v[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + q * THREADS;
    const int jj = idx / NB, ii = idx - jj * NB;          // lanes along rows
    const int i = k0 + ii, j = c0 + jj;
    if (idx < NB * NB && ii < kw && jj < cw && j - i <= ku && i - j <= kl) US[usl_idx(i, j, ku)] = Ub[ii * SP + jj];
  }
}

// Inverse of the unit lower triangle of a factored diagonal block (rows 0..NB-1 of the panel
// in Pn, row stride SP), by warp 0 (lane j: column j, by substitution in registers), into Li
// (shared, column-major with column stride SP, so that the lanes' stores fall in different
// banks) and then, lanes along rows, into dli (global, column-major NB x NB, coalesced).
// (The inverse of the upper triangle, which only the solves need, is formed afterwards from
// the diagonal block kept in the band.)
template <typename T>
__device__ void unit_lower_inverse(const T* __restrict__ Pn, int kw, T* __restrict__ Li, T* __restrict__ dli) {
  constexpr int NB = LU_NB;
  const int j = threadIdx.x;
  if (j < NB) {
    T x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      T v = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int p = 0; p < i; ++p) v -= Pn[i * SP + p] * x[p];
      x[i] = (i < kw) ? v : T(0);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) Li[j * SP + i] = x[i];
    __syncwarp();
#pragma unroll 4
    for (int c = 0; c < NB; ++c) dli[c * NB + j] = Li[c * SP + j];
  }
}

// acc[0..W) -= sum_p l(p) Uv[p][c0 .. c0+W)  (Uv row-major NB x NB, broadcast vector reads);
// the loop over p is fully unrolled so that l(p) may read a register array.
template <typename T, int W, typename LF>
__device__ __forceinline__ void row_update(T (&acc)[W], LF lf, const T* __restrict__ Uv, int c0) {
  constexpr int NB = LU_NB;
#pragma unroll
  for (int p = 0; p < NB; ++p) {
    const T l = lf(p);
    if constexpr (sizeof(T) == 4) {
      const float4* u = reinterpret_cast<const float4*>(Uv + p * NB + c0);
#pragma unroll
      for (int c4 = 0; c4 < W / 4; ++c4) {
        const float4 v = u[c4];
        acc[4 * c4 + 0] -= l * v.x;
        acc[4 * c4 + 1] -= l * v.y;
        acc[4 * c4 + 2] -= l * v.z;
        acc[4 * c4 + 3] -= l * v.w;
      }
    } else {
      const double2* u = reinterpret_cast<const double2*>(Uv + p * NB + c0);
#pragma unroll
      for (int c2 = 0; c2 < W / 2; ++c2) {
        const double2 v = u[c2];
        acc[2 * c2 + 0] -= l * v.x;
        acc[2 * c2 + 1] -= l * v.y;
      }
    }
  }
}

// Tensor-core trailing update (TPNS_TF32_IR): mma.sync m16n8k8 with TF32 operands and FP32
// accumulation; each operand is split as x = hi + lo (hi, lo TF32) and the product taken as
// hi*hi + hi*lo + lo*hi, which keeps the update close to FP32 accuracy (the error-compensated
// split of Ootomo and Yokota, 2022).
__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A22(rows rb..rb+31, columns cs..cs+15) -= L21 U12 on the tensor cores, one warp: the tile
// is 2 x 2 fragments of 16 x 8 (rows g, g+8 and columns 2t, 2t+1 of each, g = lane / 4,
// t = lane % 4); L(r, k0 + q) = Ls[q kl + r - q - 1] inside the band, U12 = Uv (row-major).
static __device__ void tc_update_tile(float* __restrict__ AB, const float* __restrict__ Ls, const float* __restrict__ Uv,
                               int k0, int kw, int R, int rb, int c0, int cw, int cs, int hcol, int kl, int ku,
                               int ldab) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float c[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e >> 1) * 8, j = cs + nt * 8 + 2 * t + (e & 1), i = k0 + r;
        c[mt][nt][e] = (r < R && j < c0 + cw && i - j <= kl && j - i <= ku)
                           ? __ldcg(AB + (int64_t)j * ldab + (ku + i - j)) : 0.0f;
      }
#pragma unroll
  for (int kk = 0; kk < LU_NB; kk += 8) {
    unsigned ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e & 1) * 8, q = kk + t + (e >> 1) * 4, o = r - q - 1;
        const float val = (r < R && q < kw && o >= 0 && o < kl) ? -Ls[q * kl + o] : 0.0f;
        split_tf32(val, ah[mt][e], al[mt][e]);
      }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float val = Uv[(kk + t + e * 4) * LU_NB + hcol + nt * 8 + g];
        split_tf32(val, bh[nt][e], bl[nt][e]);
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        mma_tf32(c[mt][nt], al[mt], bh[nt]);
        mma_tf32(c[mt][nt], ah[mt], bl[nt]);
        mma_tf32(c[mt][nt], ah[mt], bh[nt]);
      }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e >> 1) * 8, j = cs + nt * 8 + 2 * t + (e & 1), i = k0 + r;
        if (r < R && j < c0 + cw && i - j <= kl && j - i <= ku) AB[(int64_t)j * ldab + (ku + i - j)] = c[mt][nt][e];
      }
}

// The same tile in plain BF16 (TPNS_BF16_IR): mma.sync m16n8k16 with BF16 operands (each value
// rounded once) and FP32 accumulation; the factors then carry BF16-level error, which the
// FP64-residual refinement has to win back.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
static __device__ void tc_update_tile_bf16(float* __restrict__ AB, const float* __restrict__ Ls,
                                           const float* __restrict__ Uv, int k0, int kw, int R, int rb, int c0, int cw,
                                           int cs, int hcol, int kl, int ku, int ldab) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float c[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e >> 1) * 8, j = cs + nt * 8 + 2 * t + (e & 1), i = k0 + r;
        c[mt][nt][e] = (r < R && j < c0 + cw && i - j <= kl && j - i <= ku)
                           ? __ldcg(AB + (int64_t)j * ldab + (ku + i - j)) : 0.0f;
      }
  auto lval = [&](int r, int q) -> float {
    const int o = r - q - 1;
    return (r < R && q < kw && o >= 0 && o < kl) ? -Ls[q * kl + o] : 0.0f;
  };
#pragma unroll
  for (int kk = 0; kk < LU_NB; kk += 16) {
    unsigned a[2][4], b[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e & 1) * 8, q = kk + 2 * t + (e >> 1) * 8;
        a[mt][e] = pack_bf16(lval(r, q), lval(r, q + 1));
      }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int q = kk + 2 * t + e * 8, col = hcol + nt * 8 + g;
        b[nt][e] = pack_bf16(Uv[q * LU_NB + col], Uv[(q + 1) * LU_NB + col]);
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) mma_bf16(c[mt][nt], a[mt], b[nt]);
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = rb + mt * 16 + g + (e >> 1) * 8, j = cs + nt * 8 + 2 * t + (e & 1), i = k0 + r;
        if (r < R && j < c0 + cw && i - j <= kl && j - i <= ku) AB[(int64_t)j * ldab + (ku + i - j)] = c[mt][nt][e];
      }
}

template <typename T, bool WIDE, int CL, int TC>
__global__ void __launch_bounds__(lu_threads<T>(), 1)
band_lu_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list, T* __restrict__ band,
               T* __restrict__ lslab, T* __restrict__ uslab, T* __restrict__ dinv_all, int* __restrict__ sync_all,
               int sync_stride, const int* __restrict__ epoch_ptr, int* __restrict__ status, const int* skip) {
  if (skip && *skip) return;
  const int epoch = *epoch_ptr;   // this factorisation's tag for the panel flags and counters
  constexpr int NB = LU_NB;
  constexpr int THREADS = lu_threads<T>();
  constexpr int HALF = NB / 2;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  constexpr int nbulk = CL - 1;
  const int sid = list[blockIdx.x / CL];
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku, ldab = S.ldab;
  T* AB = band + S.band_off;
  T* LS = lslab + S.lslab_off;
  T* US = uslab + S.uslab_off;
  T* DI = dinv_all + S.dinv_off;
  int* flag = sync_all + (int64_t)sid * sync_stride;
  int* cnt = flag + sync_stride / 2;
  int* st = status + sid;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);     // one mbarrier (bulk CTAs)
  T* Uv = reinterpret_cast<T*>(smem_raw + 128);              // NB x NB
  T* Li = Uv + NB * NB;                                      // L11^{-1} column-major: NB x SP (critical),
                                                             // NB x NB by TMA (bulk)
  T* Ub = Li + NB * SP;                                      // NB x SP
  T* prow = Ub + NB * SP;                                    // NB x PR pivot rows (16-byte aligned)
  T* Pn = prow + NB * PR;                                    // critical, wide: (NB + kl) x SP panel
  T* Dt = prow + NB * PR;                                    // critical: NB x SP diagonal block
  T* Lsk = Dt + NB * SP;                                     // critical: NB x kl skewed L (16-byte aligned)
  T* Ls = prow;                                              // bulk: NB x kl L slab (16-byte aligned)
  __shared__ int abort_flag;
  const int nblk = (n + NB - 1) / NB;
  const int D = (31 + ku) / 32;                              // blocks right of a panel inside its window
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = THREADS / 32;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (WIDE && rank == 0) {
    // ------------------------------------------------ critical CTA, panels taller than the CTA:
    // the panel stays in shared memory and every thread works on rows tid, tid + THREADS, ...
    {
      const int kw = min(NB, n), R = min(n, kw + kl);
      for (int r = tid; r < R; r += THREADS) {
#pragma unroll 4
        for (int c = 0; c < NB; ++c)
          Pn[r * SP + c] = (c < kw && r - c <= kl && c - r <= ku) ? __ldcg(AB + (int64_t)c * ldab + (ku + r - c)) : T(0);
      }
      __syncthreads();
      factor_panel_smem<T>(0, kw, R, kl, ku, ldab, AB, LS, US, Pn, prow, st);
      __syncthreads();
      unit_lower_inverse<T>(Pn, kw, Li, DI);
      __syncthreads();
      if (tid == 0) st_release(flag + 0, epoch);
    }
    const int nslice = (NB + kl + THREADS - 1) / THREADS;
    for (int kb = 0; kb + 1 < nblk; ++kb) {
      const int k0 = kb * NB, R = min(n, k0 + NB + kl) - k0;
      const int cb = kb + 1, c0 = cb * NB, cw = min(NB, n - c0), R2 = min(n, c0 + cw + kl) - c0;
      const int need = cb - 1 - max(0, cb - D);
      if (need > 0 && tid == 0) {
        if (!wait_cnt(cnt + cb, epoch, need)) {
          atomicOr(st, 2);
          abort_flag = 1;
        }
      }
      __syncthreads();
      if (abort_flag) return;
      form_u12<T>(Li, SP, Ub, Uv, AB, US, k0, NB, c0, cw, kl, ku, ldab);
      // rows of the next panel, updated by this panel, in slices of THREADS rows: row r2 reads
      // row r2 + NB of this panel, so a slice is written back only after all its reads
      for (int q = 0; q < nslice; ++q) {
        const int r2 = q * THREADS + tid, i = c0 + r2, r = r2 + NB;
        T a[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const int j = c0 + c;
          a[c] = (r2 < R2 && c < cw && i - j <= kl && j - i <= ku) ? __ldcg(AB + (int64_t)j * ldab + (ku + i - j)) : T(0);
        }
        if (r2 < R2 && r < R) row_update<T, NB>(a, [&](int p) { return Pn[r * SP + p]; }, Uv, 0);
        __syncthreads();
        if (r2 < R2) {
#pragma unroll
          for (int c = 0; c < NB; ++c) Pn[r2 * SP + c] = a[c];
        }
      }
      __syncthreads();
      factor_panel_smem<T>(c0, cw, R2, kl, ku, ldab, AB, LS, US, Pn, prow, st);
      __syncthreads();
      unit_lower_inverse<T>(Pn, cw, Li, DI + (int64_t)cb * 2 * NB * NB);
      __syncthreads();
      if (tid == 0) st_release(flag + cb, epoch);
    }
  } else if (rank == 0) {
    // ------------------------------------------------ critical CTA: the chain of panels
    T a[NB];
    {
      const int kw = min(NB, n), R = min(n, kw + kl), r = tid;
#pragma unroll
      for (int c = 0; c < NB; ++c)
        a[c] = (r < R && c < kw && r - c <= kl && c - r <= ku) ? __ldcg(AB + (int64_t)c * ldab + (ku + r - c)) : T(0);
      factor_rows<T>(a, 0, kw, R, kl, ku, ldab, AB, US, Dt, Lsk, prow, st);
      __syncthreads();
      if (tid == 0) tma_store_lslab(LS, Lsk, kl);
      unit_lower_inverse<T>(Dt, kw, Li, DI);
      __syncthreads();
      if (tid == 0) {
        tma_store_wait();
        st_release(flag + 0, epoch);   // release orders the CTA's writes (after the barrier)
      }
    }
    for (int kb = 0; kb + 1 < nblk; ++kb) {
      const int k0 = kb * NB, R = min(n, k0 + NB + kl) - k0;
      const int cb = kb + 1, c0 = cb * NB, cw = min(NB, n - c0), R2 = min(n, c0 + cw + kl) - c0;
      const int need = cb - 1 - max(0, cb - D);
      if (need > 0 && tid == 0) {
        if (!wait_cnt(cnt + cb, epoch, need)) {
          atomicOr(st, 2);
          abort_flag = 1;
        }
      }
      __syncthreads();
      if (abort_flag) return;
      form_u12<T>(Li, SP, Ub, Uv, AB, US, k0, NB, c0, cw, kl, ku, ldab);
      // the row of the next panel held by this thread, updated by this panel on the way in
      {
        const int r2 = tid, i = c0 + r2, r = r2 + NB;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const int j = c0 + c;
          a[c] = (r2 < R2 && c < cw && i - j <= kl && j - i <= ku) ? __ldcg(AB + (int64_t)j * ldab + (ku + i - j)) : T(0);
        }
        // L(r, p) of this panel, zero outside the band
        if (r2 < R2 && r < R)
          row_update<T, NB>(a, [&](int p) { return r - p - 1 < kl ? Lsk[p * kl + (r - p - 1)] : T(0); }, Uv, 0);
      }
      __syncthreads();
      factor_rows<T>(a, c0, cw, R2, kl, ku, ldab, AB, US, Dt, Lsk, prow, st);
      __syncthreads();
      if (tid == 0) tma_store_lslab(LS + (int64_t)cb * NB * kl, Lsk, kl);
      unit_lower_inverse<T>(Dt, cw, Li, DI + (int64_t)cb * 2 * NB * NB);
      __syncthreads();
      if (tid == 0) {
        tma_store_wait();
        st_release(flag + cb, epoch);
      }
    }
  } else {
    // ------------------------------------------------ bulk CTAs: blocks p+2 .. of every panel p
    int uses = 0;
    for (int p = 0; p < nblk; ++p) {
      const int k0 = p * NB, kw = min(NB, n - k0), R = min(n, k0 + kw + kl) - k0;
      const int cbl = min(nblk - 1, (k0 + kw - 1 + ku) / NB);
      int first = p + 2;
      while (first <= cbl && 1 + first % nbulk != rank) ++first;
      if (first > cbl) continue;
      if (tid == 0) {
        bool ok = wait_eq(flag + p, epoch);
        if (ok) {
          // the panel's L slab and L11^{-1}, written by CTA 0, by TMA into shared memory
          asm volatile("fence.proxy.async.global;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const unsigned bl = (unsigned)(NB * kl * sizeof(T)), bi = (unsigned)(NB * NB * sizeof(T));
          mbar_expect_tx(bar, bl + bi);
          tma_bulk_g2s(Li, DI + (int64_t)p * 2 * NB * NB, bi, bar);
          if (bl) tma_bulk_g2s(Ls, LS + (int64_t)p * NB * kl, bl, bar);
          int it = 0;
          while (!mbar_try_wait(bar, (unsigned)(uses & 1))) {
            if (++it > WAIT_LIMIT) {
              ok = false;
              break;
            }
          }
        }
        if (!ok) {
          atomicOr(st, 2);
          abort_flag = 1;
        }
      }
      ++uses;
      __syncthreads();
      if (abort_flag) return;
      for (int cb = first; cb <= cbl; cb += nbulk) {
        const int c0 = cb * NB, cw = min(NB, n - c0);
        form_u12<T>(Li, NB, Ub, Uv, AB, US, k0, kw, c0, cw, kl, ku, ldab);
        // A22 -= L21 U12: warp pairs share 32 rows (lane = row), each warp one half of the columns
        const int h = warp & 1, groups = nwarp / 2;
        if constexpr (TC == 1 && sizeof(T) == 4) {
          for (int rb = kw + (warp >> 1) * 32; rb < R; rb += groups * 32)
            tc_update_tile(reinterpret_cast<float*>(AB), reinterpret_cast<const float*>(Ls),
                           reinterpret_cast<const float*>(Uv), k0, kw, R, rb, c0, cw, c0 + h * HALF, h * HALF, kl, ku,
                           ldab);
        } else if constexpr (TC == 2 && sizeof(T) == 4) {
          for (int rb = kw + (warp >> 1) * 32; rb < R; rb += groups * 32)
            tc_update_tile_bf16(reinterpret_cast<float*>(AB), reinterpret_cast<const float*>(Ls),
                                reinterpret_cast<const float*>(Uv), k0, kw, R, rb, c0, cw, c0 + h * HALF, h * HALF, kl,
                                ku, ldab);
        } else
        for (int rb = kw + (warp >> 1) * 32; rb < R; rb += groups * 32) {
          const int r = rb + lane;
          if (r < R) {
            const int i = k0 + r;
            const int cs = c0 + h * HALF;
            T acc[HALF];
            T* a0 = AB + (int64_t)cs * ldab + (ku + i - cs);    // A(i, cs + jj) = a0[jj * (ldab - 1)]
#pragma unroll
            for (int jj = 0; jj < HALF; ++jj) {
              const int j = cs + jj;
              acc[jj] = (j < c0 + cw && i - j <= kl && j - i <= ku) ? __ldcg(a0 + (int64_t)jj * (ldab - 1)) : T(0);
            }
            // L(i, k0 + q) = Ls[q * kl + (r - q - 1)] for 0 <= r - q - 1 < kl
            row_update<T, HALF>(acc, [&](int q) {
              const int o = r - q - 1;
              return (q < kw && o < kl) ? Ls[q * kl + o] : T(0);
            }, Uv, h * HALF);
#pragma unroll
            for (int jj = 0; jj < HALF; ++jj) {
              const int j = cs + jj;
              if (j < c0 + cw && i - j <= kl && j - i <= ku) a0[(int64_t)jj * (ldab - 1)] = acc[jj];
            }
          }
        }
        __syncthreads();
        if (tid == 0) st_release(cnt + cb, cnt_word(epoch, p - max(0, cb - D) + 1));
      }
    }
  }
}

// Dynamic shared memory of the LU kernel: mbarrier (128 B), Uv (NB x NB), Li and Ub
// (NB x SP each), then the larger of the chain CTA's part [pivot rows NB x PR, then the
// diagonal block NB x SP and the skewed L buffer NB x kl, or (wide) the panel (NB + kl) x SP]
// and the bulk CTAs' L slab NB x kl.
template <typename T>
size_t band_lu_smem_bytes(int kl_max) {
  const size_t head = (size_t)LU_NB * LU_NB + 2 * LU_NB * SP;
  const bool wide = LU_NB + kl_max > lu_threads<T>();
  const size_t chain = wide ? (size_t)LU_NB * PR + (size_t)(LU_NB + kl_max) * SP
                            : (size_t)LU_NB * PR + (size_t)LU_NB * SP + (size_t)LU_NB * kl_max;
  const size_t tail = std::max(chain, (size_t)LU_NB * kl_max);
  return 128 + (head + tail) * sizeof(T);
}

// a new tag for the next factorisation (kept on the device so that a captured graph replays
// with fresh tags)
static __global__ void bump_kernel(int* p) { *p = (*p % 0x7FFFF) + 1; }

template <typename T>
cudaError_t launch_band_lu(const SysDev* sys, const int* list, int nsys, int kl_max, T* band, T* lslab, T* uslab,
                           T* dinv, int* sync, int sync_stride, int* epoch, int* status, cudaStream_t st,
                           const int* skip, int tc, int cl_force) {
  if (nsys == 0) return cudaSuccess;
  const size_t smem = band_lu_smem_bytes<T>(kl_max);
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (kl_max < 0 || smem > (size_t)smem_max) return cudaErrorInvalidValue;
  // panels of at most one row per thread are factored from registers
  const bool wide = LU_NB + kl_max > lu_threads<T>();
  auto kern8 = wide ? band_lu_kernel<T, true, LU_CLUSTER, 0> : band_lu_kernel<T, false, LU_CLUSTER, 0>;
  auto kern16 = wide ? band_lu_kernel<T, true, 2 * LU_CLUSTER, 0> : band_lu_kernel<T, false, 2 * LU_CLUSTER, 0>;
  if constexpr (sizeof(T) == 4) {
    if (tc == 1) {
      kern8 = wide ? band_lu_kernel<T, true, LU_CLUSTER, 1> : band_lu_kernel<T, false, LU_CLUSTER, 1>;
      kern16 = wide ? band_lu_kernel<T, true, 2 * LU_CLUSTER, 1> : band_lu_kernel<T, false, 2 * LU_CLUSTER, 1>;
    } else if (tc == 2) {
      kern8 = wide ? band_lu_kernel<T, true, LU_CLUSTER, 2> : band_lu_kernel<T, false, LU_CLUSTER, 2>;
      kern16 = wide ? band_lu_kernel<T, true, 2 * LU_CLUSTER, 2> : band_lu_kernel<T, false, 2 * LU_CLUSTER, 2>;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kern8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(lu_threads<T>(), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // very wide bands (or cl_force = 16): 16-CTA clusters (15 CTAs on the trailing updates)
  // when all of them fit on the device at once and it can place them, else 8
  int cl = LU_CLUSTER, nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool want16 = cl_force == 2 * LU_CLUSTER || (cl_force == 0 && kl_max > LU_WIDE_CLUSTER_KL);
  if (want16 && nsys * 2 * LU_CLUSTER <= nsm &&
      cudaFuncSetAttribute(kern16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
      cudaFuncSetAttribute(kern16, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    int nclusters = 0;
    attr[0].val.clusterDim.x = 2 * LU_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * LU_CLUSTER, 1, 1);
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern16, &cfg) == cudaSuccess && nclusters > 0) cl = 2 * LU_CLUSTER;
    cudaGetLastError();
  }
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(nsys * cl, 1, 1);
  count_launches(2);
  bump_kernel<<<1, 1, 0, st>>>(epoch);
  e = cudaLaunchKernelEx(&cfg, cl == LU_CLUSTER ? kern8 : kern16, sys, list, band, lslab, uslab, dinv, sync, sync_stride, (const int*)epoch, status,
                         skip);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Diagonal-block inverses of a factored unit-L / U band: one CTA per (block, system).
template <typename T>
__global__ void __launch_bounds__(64) band_dinv_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                      const T* __restrict__ band, T* __restrict__ dinv_all,
                                                      const int* skip) {
  if (skip && *skip) return;
  constexpr int NB = LU_NB;
  const SysDev S = sys[list[blockIdx.y]];
  const int nblk = (S.n + NB - 1) / NB;
  const int kb = blockIdx.x;
  if (kb >= nblk) return;
  const T* AB = band + S.band_off;
  __shared__ T D[NB * SP];
  const int k0 = kb * NB, kw = min(NB, S.n - k0);
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int c = idx / NB, r = idx - c * NB;
    const int i = k0 + r, j = k0 + c;
    D[r * SP + c] = (r < kw && c < kw && i - j <= S.kl && j - i <= S.ku) ? AB[(int64_t)j * S.ldab + (S.ku + i - j)] : T(0);
  }
  __syncthreads();
  diag_inverses<T>(D, kw, dinv_all + S.dinv_off + (int64_t)kb * 2 * NB * NB);
}

template <typename T>
cudaError_t launch_band_dinv(const SysDev* sys, const int* list, int nsys, int nblk_max, const T* band, T* dinv,
                             cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  band_dinv_kernel<T><<<dim3(nblk_max, nsys), 64, 0, st>>>(sys, list, band, dinv, skip);
  return cudaGetLastError();
}

// Slabs of an already factored band (used once for the Darcy factors).
template <typename T>
__global__ void band_to_slab_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                    const T* __restrict__ band, T* __restrict__ lslab, T* __restrict__ uslab) {
  const SysDev S = sys[list[blockIdx.y]];
  const T* AB = band + S.band_off;
  const int64_t tot = (int64_t)S.n * S.ldab;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / S.ldab), off = (int)(idx % S.ldab);
    const int i = off - S.ku + j;
    if (i < 0 || i >= S.n) continue;
    if (i > j) lslab[S.lslab_off + lsl_idx(i, j, S.kl)] = AB[idx];
    else if (i < j) uslab[S.uslab_off + usl_idx(i, j, S.ku)] = AB[idx];
  }
}

template <typename T>
cudaError_t launch_band_to_slab(const SysDev* sys, const int* list, int nsys, const T* band, T* lslab, T* uslab,
                                cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  band_to_slab_kernel<T><<<dim3(64, nsys), 256, 0, st>>>(sys, list, band, lslab, uslab);
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
// x (+)= U^{-1} L^{-1} r for unit-lower L and upper U, one CTA per system.  The factors are
// read from the per-block slabs: every block's slab (32 columns x kl or ku rows, contiguous)
// and the inverse of its diagonal triangle arrive in shared memory with two TMA bulk copies
// completing on an mbarrier, STAGES blocks ahead of the one being solved.  Each block is
// finished by one warp with the inverse (a GEMV), then the rows coupled to it by the band are
// updated by all threads.  The vector lives in shared memory in precision T.
constexpr int SOLVE_THREADS = 512;

template <typename T, int STAGES, bool GV>
__global__ void __launch_bounds__(SOLVE_THREADS) band_solve_kernel(const SysDev* __restrict__ sys,
                                                         const int* __restrict__ list,
                                                         const T* __restrict__ lslab, const T* __restrict__ uslab,
                                                         const T* __restrict__ dinv_all,
                                                         const double* __restrict__ rhs,
                                                         double* __restrict__ x, int accumulate, int kmax,
                                                         const int* __restrict__ done, int* __restrict__ status,
                                                         const int* skip, T* __restrict__ vwork) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.x];
  if (done && done[sid]) return;
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku;
  constexpr int NB = LU_NB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);                  // STAGES mbarriers
  T* stage0 = reinterpret_cast<T*>(smem_raw + 128);
  const size_t stage_elems = (size_t)NB * NB + (size_t)NB * kmax;         // inverse, then slab
  // the vector: in shared memory after the stages, or (GV) in the caller's global scratch
  // at the system's offset when it does not fit
  T* v = GV ? vwork + S.x_off : stage0 + STAGES * stage_elems;
  __shared__ T yb[NB];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + NB - 1) / NB;
  const int total = 2 * nblk;                                             // forward then backward
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < STAGES; ++k) mbar_init(bar + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const double* b = rhs + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) v[i] = (T)b[i];
  __syncthreads();
  auto issue = [&](int g) {   // thread 0 only
    const int s = g % STAGES;
    const bool fwd = g < nblk;
    const int kb = fwd ? g : 2 * nblk - 1 - g;
    const int w = fwd ? kl : ku;
    T* dst = stage0 + s * stage_elems;
    const T* di = dinv_all + S.dinv_off + (int64_t)kb * 2 * NB * NB + (fwd ? 0 : NB * NB);
    const T* sl = (fwd ? lslab + S.lslab_off : uslab + S.uslab_off) + (int64_t)kb * NB * w;
    const unsigned bi = NB * NB * sizeof(T), bs = (unsigned)(NB * w * sizeof(T));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar + s, bi + bs);
    tma_bulk_g2s(dst, di, bi, bar + s);
    if (bs) tma_bulk_g2s(dst + NB * NB, sl, bs, bar + s);
  };
  if (tid == 0)
    for (int g = 0; g < STAGES && g < total; ++g) issue(g);
  for (int g = 0; g < total; ++g) {
    const int s = g % STAGES;
    const unsigned parity = (unsigned)((g / STAGES) & 1);
    if (tid == 0) {
      int it = 0;
      while (!mbar_try_wait(bar + s, parity)) {
        if (++it > WAIT_LIMIT) {
          atomicOr(status + sid, 2);
          abort_flag = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (abort_flag) {
      // let the copies already issued land before leaving (bounded)
      if (tid == 0)
        for (int h = g + 1; h < g + STAGES && h < total; ++h)
          for (int it = 0; !mbar_try_wait(bar + h % STAGES, (unsigned)((h / STAGES) & 1)) && it < WAIT_LIMIT; ++it) {
          }
      return;
    }
    const bool fwd = g < nblk;
    const int kb = fwd ? g : 2 * nblk - 1 - g;
    const int k0 = kb * NB, kw = min(NB, n - k0);
    const int w = fwd ? kl : ku;
    const T* Dv = stage0 + s * stage_elems;
    const T* sl = Dv + NB * NB;
    if (warp == 0) {
      // four partial sums: short dependency chains
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int p = 0; p < NB; ++p)
        if (p < kw) acc[p & 3] += Dv[p * NB + lane] * v[k0 + p];
      yb[lane] = lane < kw ? (acc[0] + acc[1]) + (acc[2] + acc[3]) : T(0);
    }
    __syncthreads();
    if (tid < kw) v[k0 + tid] = yb[tid];
    if (fwd) {
      const int rend = min(n, k0 + kw + kl);
      for (int i = k0 + kw + tid; i < rend; i += blockDim.x) {
        // L(i, k0 + c) = sl[c * kl + (i - k0 - c - 1)], valid for 0 <= i - k0 - c - 1 < kl;
        // four partial sums
        const int ob = i - k0 - 1;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < kw && ob - c < kl) acc[c & 3] += sl[c * w + (ob - c)] * yb[c];
        v[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
      }
    } else {
      const int rbeg = max(0, k0 - ku);
      for (int i = rbeg + tid; i < k0; i += blockDim.x) {
        // U(i, k0 + c) = sl[c * ku + (i - k0 - c + ku)], valid for 0 <= i - k0 - c + ku
        const int ob = i - k0 + ku;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < kw && ob - c >= 0) acc[c & 3] += sl[c * w + (ob - c)] * yb[c];
        v[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
      }
    }
    __syncthreads();
    if (tid == 0 && g + STAGES < total) issue(g + STAGES);
  }
  double* xo = x + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) xo[i] = accumulate ? xo[i] + (double)v[i] : (double)v[i];
}

// true if one CTA holds the vector of n_max entries and at least one pipeline stage
template <typename T>
bool band_solve_fits_smem(int n_max, int kmax) {
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t stage = ((size_t)LU_NB * LU_NB + (size_t)LU_NB * kmax) * sizeof(T);
  return 128 + stage + ((size_t)n_max + 4) * sizeof(T) + 1024 <= (size_t)smem_max;
}

// The solve for systems whose vector lives in global scratch (too large for shared memory):
// blocks are streamed in halves (diagonal inverse + slab columns 0..15, then columns
// 16..31) through HS half-stages, so that several halves are in flight even for the widest
// bands; each half's band updates run as soon as it lands.  Otherwise as band_solve_kernel.
template <typename T, int HS>
__global__ void __launch_bounds__(SOLVE_THREADS) band_solve_halves_kernel(
    const SysDev* __restrict__ sys, const int* __restrict__ list, const T* __restrict__ lslab,
    const T* __restrict__ uslab, const T* __restrict__ dinv_all, const double* __restrict__ rhs, double* __restrict__ x,
    int accumulate, int kmax, const int* __restrict__ done, int* __restrict__ status, const int* skip,
    T* __restrict__ vwork) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.x];
  if (done && done[sid]) return;
  const SysDev S = sys[sid];
  const int n = S.n, kl = S.kl, ku = S.ku;
  constexpr int NB = LU_NB, HB = LU_NB / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);                  // HS mbarriers
  T* stage0 = reinterpret_cast<T*>(smem_raw + 128);
  const size_t stage_elems = (size_t)NB * NB + (size_t)HB * kmax;         // inverse, half slab
  T* v = vwork + S.x_off;
  __shared__ T yb[NB];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + NB - 1) / NB;
  const int total = 4 * nblk;                                             // halves, forward then backward
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < HS; ++k) mbar_init(bar + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const double* b = rhs + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) v[i] = (T)b[i];
  __syncthreads();
  auto issue = [&](int h) {   // thread 0 only
    const int s = h % HS, g = h >> 1, half = h & 1;
    const bool fwd = g < nblk;
    const int kb = fwd ? g : 2 * nblk - 1 - g;
    const int w = fwd ? kl : ku;
    T* dst = stage0 + s * stage_elems;
    const T* di = dinv_all + S.dinv_off + (int64_t)kb * 2 * NB * NB + (fwd ? 0 : NB * NB);
    const T* sl = (fwd ? lslab + S.lslab_off : uslab + S.uslab_off) + (int64_t)kb * NB * w + (int64_t)half * HB * w;
    const unsigned bi = half ? 0u : (unsigned)(NB * NB * sizeof(T)), bs = (unsigned)(HB * w * sizeof(T));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar + s, bi + bs);
    if (bi) tma_bulk_g2s(dst, di, bi, bar + s);
    if (bs) tma_bulk_g2s(dst + NB * NB, sl, bs, bar + s);
  };
  if (tid == 0)
    for (int h = 0; h < HS && h < total; ++h) issue(h);
  for (int g = 0; g < 2 * nblk; ++g) {
    const bool fwd = g < nblk;
    const int kb = fwd ? g : 2 * nblk - 1 - g;
    const int k0 = kb * NB, kw = min(NB, n - k0);
    const int w = fwd ? kl : ku;
    for (int half = 0; half < 2; ++half) {
      const int h = 2 * g + half, s = h % HS;
      if (tid == 0) {
        int it = 0;
        while (!mbar_try_wait(bar + s, (unsigned)((h / HS) & 1))) {
          if (++it > WAIT_LIMIT) {
            atomicOr(status + sid, 2);
            abort_flag = 1;
            break;
          }
        }
      }
      __syncthreads();
      if (abort_flag) {
        if (tid == 0)
          for (int q = h + 1; q < h + HS && q < total; ++q)
            for (int it = 0; !mbar_try_wait(bar + q % HS, (unsigned)((q / HS) & 1)) && it < WAIT_LIMIT; ++it) {
            }
        return;
      }
      const T* Dv = stage0 + s * stage_elems;
      const T* sl = Dv + NB * NB;
      if (half == 0) {
        if (warp == 0) {
          T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int p = 0; p < NB; ++p)
            if (p < kw) acc[p & 3] += Dv[p * NB + lane] * v[k0 + p];
          yb[lane] = lane < kw ? (acc[0] + acc[1]) + (acc[2] + acc[3]) : T(0);
        }
        __syncthreads();
        if (tid < kw) v[k0 + tid] = yb[tid];
      }
      const int cb0 = half * HB;
      if (fwd) {
        const int rend = min(n, k0 + kw + kl);
        for (int i = k0 + kw + tid; i < rend; i += blockDim.x) {
          const int ob = i - k0 - 1;
          T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int cc = 0; cc < HB; ++cc) {
            const int c = cb0 + cc;
            if (c < kw && ob - c < kl) acc[cc & 3] += sl[cc * w + (ob - c)] * yb[c];
          }
          v[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
      } else {
        const int rbeg = max(0, k0 - ku);
        for (int i = rbeg + tid; i < k0; i += blockDim.x) {
          const int ob = i - k0 + ku;
          T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int cc = 0; cc < HB; ++cc) {
            const int c = cb0 + cc;
            if (c < kw && ob - c >= 0) acc[cc & 3] += sl[cc * w + (ob - c)] * yb[c];
          }
          v[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
      }
      __syncthreads();
      if (tid == 0 && h + HS < total) issue(h + HS);
    }
  }
  double* xo = x + S.x_off;
  for (int i = tid; i < n; i += blockDim.x) xo[i] = accumulate ? xo[i] + (double)v[i] : (double)v[i];
}

template <typename T, int HS>
static cudaError_t launch_solve_halves(size_t smem, const SysDev* sys, const int* list, int nsys, int kmax,
                                       const T* lslab, const T* uslab, const T* dinv, const double* r, double* x,
                                       int accumulate, const int* done, int* status, cudaStream_t st,
                                       const int* skip, T* vwork) {
  cudaError_t e = cudaFuncSetAttribute(band_solve_halves_kernel<T, HS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  band_solve_halves_kernel<T, HS><<<nsys, SOLVE_THREADS, smem, st>>>(sys, list, lslab, uslab, dinv, r, x, accumulate,
                                                                     kmax, done, status, skip, vwork);
  return cudaGetLastError();
}

template <typename T, int STAGES, bool GV>
static cudaError_t launch_solve_variant(size_t smem, const SysDev* sys, const int* list, int nsys, int kmax,
                                        const T* lslab, const T* uslab, const T* dinv, const double* r, double* x,
                                        int accumulate, const int* done, int* status, cudaStream_t st,
                                        const int* skip, T* vwork) {
  cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<T, STAGES, GV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  band_solve_kernel<T, STAGES, GV><<<nsys, SOLVE_THREADS, smem, st>>>(sys, list, lslab, uslab, dinv, r, x, accumulate, kmax,
                                                            done, status, skip, vwork);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_solve(const SysDev* sys, const int* list, int nsys, int n_max, int kmax, const T* lslab,
                              const T* uslab, const T* dinv, const double* r, double* x, int accumulate,
                              const int* done, int* status, cudaStream_t st, const int* skip, T* vwork) {
  if (nsys == 0) return cudaSuccess;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t stage = ((size_t)LU_NB * LU_NB + (size_t)LU_NB * kmax) * sizeof(T);
  const size_t vec = ((size_t)n_max + 4) * sizeof(T);
  const size_t static_smem = 1024;
  count_launches(1);
  // deepest pipeline with the vector in shared memory, else (given scratch) the vector in
  // global memory with half-block stages, else with whole-block stages
  if (vwork && !band_solve_fits_smem<T>(n_max, kmax)) {
    const size_t half = ((size_t)LU_NB * LU_NB + (size_t)(LU_NB / 2) * kmax) * sizeof(T);
    for (int hs = 3; hs >= 2; --hs) {
      const size_t need = 128 + hs * half;
      if (need + static_smem > (size_t)smem_max) continue;
      if (hs == 3)
        return launch_solve_halves<T, 3>(need, sys, list, nsys, kmax, lslab, uslab, dinv, r, x, accumulate, done,
                                         status, st, skip, vwork);
      return launch_solve_halves<T, 2>(need, sys, list, nsys, kmax, lslab, uslab, dinv, r, x, accumulate, done,
                                       status, st, skip, vwork);
    }
  }
  for (int gv = 0; gv < 2; ++gv) {
    if (gv && !vwork) break;
    for (int stages = 3; stages >= 1; --stages) {
      const size_t need = 128 + stages * stage + (gv ? 0 : vec);
      if (need + static_smem > (size_t)smem_max) continue;
#define TPNS_SOLVE_ARGS need, sys, list, nsys, kmax, lslab, uslab, dinv, r, x, accumulate, done, status, st, skip, vwork
      if (!gv) {
        if (stages == 3) return launch_solve_variant<T, 3, false>(TPNS_SOLVE_ARGS);
        if (stages == 2) return launch_solve_variant<T, 2, false>(TPNS_SOLVE_ARGS);
        return launch_solve_variant<T, 1, false>(TPNS_SOLVE_ARGS);
      }
      if (stages == 3) return launch_solve_variant<T, 3, true>(TPNS_SOLVE_ARGS);
      if (stages == 2) return launch_solve_variant<T, 2, true>(TPNS_SOLVE_ARGS);
      return launch_solve_variant<T, 1, true>(TPNS_SOLVE_ARGS);
#undef TPNS_SOLVE_ARGS
    }
  }
  count_launches(-1);
  return cudaErrorInvalidValue;
}

#if TPNS_BAND_PART == 1
// ------------------------------------------------------------------------------ residual
// r = b - A x (FP64 CSR), relative residual and refinement control.  RES_CHUNKS CTAs per
// system each handle a slice of rows and store partial sums of ||r||^2 and ||b||^2; the last
// CTA of a system to finish (atomic ticket) adds the partials in slice order, so the result
// does not depend on scheduling.  A system stops when ||r|| <= tol ||b|| or when the residual
// stagnates (||r_k|| > 0.5 ||r_{k-1}||).
__global__ void __launch_bounds__(256) residual_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                       const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colidx,
                                                       const double* __restrict__ vals,
                                                       const double* __restrict__ b, const double* __restrict__ x,
                                                       double* __restrict__ r, double* __restrict__ rel,
                                                       double* __restrict__ rel_prev, int* __restrict__ done,
                                                       int* __restrict__ iters, double* __restrict__ partial,
                                                       int* __restrict__ ticket, double tol, int first,
                                                       const int* skip) {
  if (skip && *skip) return;
  const int sid = list[blockIdx.y];
  if (!first && done[sid]) return;
  const SysDev S = sys[sid];
  const int32_t* rp = rowptr + S.rp_off;
  const int32_t* ci = colidx + S.nnz_off;
  const double* va = vals + S.val_off;
  const double* bb = b + S.x_off;
  const double* xx = x + S.x_off;
  double* rr = r + S.x_off;
  const int chunk = (S.n + RES_CHUNKS - 1) / RES_CHUNKS;
  const int r0 = blockIdx.x * chunk, r1 = min(S.n, r0 + chunk);
  double sr = 0, sb = 0;
  // four lanes per row (rows hold 10 to 50 entries), eight rows per warp at a time, so that
  // each warp keeps eight rows' dependent loads (row pointers, entries, x) in flight
  const int sl = threadIdx.x & 3, slot = threadIdx.x >> 2, per_pass = blockDim.x >> 2;
  for (int i0 = r0; i0 < r1; i0 += per_pass) {
    const int i = i0 + slot;
    double acc = 0.0;
    if (i < r1 && first != 1) {
      const int k1 = rp[i + 1];
#pragma unroll 4
      for (int k = rp[i] + sl; k < k1; k += 4) acc += va[k] * xx[ci[k]];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (sl == 0 && i < r1) {
      const double bi = bb[i], ri = bi - acc;
      rr[i] = ri;
      sr += ri * ri;
      sb += bi * bi;
    }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sr;
  red[1][threadIdx.x] = sb;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s2];
      red[1][threadIdx.x] += red[1][threadIdx.x + s2];
    }
    __syncthreads();
  }
  __shared__ int last;
  if (threadIdx.x == 0) {
    double* pp = partial + ((int64_t)sid * RES_CHUNKS + blockIdx.x) * 2;
    pp[0] = red[0][0];
    pp[1] = red[1][0];
    __threadfence();
    last = atomicAdd(ticket + sid, 1) == RES_CHUNKS - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double tr = 0, tb = 0;
  const double* pp = partial + (int64_t)sid * RES_CHUNKS * 2;
  for (int c = 0; c < RES_CHUNKS; ++c) {
    tr += __ldcg(pp + 2 * c);
    tb += __ldcg(pp + 2 * c + 1);
  }
  ticket[sid] = 0;
  const double nb = sqrt(tb);
  const double relres = nb > 0 ? sqrt(tr) / nb : 0.0;
  if (first) {
    // first == 1: x = 0, r = b; first == 2: r = b - A x for the caller's initial x, which may
    // already be converged
    iters[sid] = 0;
    rel_prev[sid] = 1.0;
    rel[sid] = nb == 0.0 ? 0.0 : (first == 2 ? relres : 1.0);
    done[sid] = (nb == 0.0 || (first == 2 && relres <= tol)) ? 1 : 0;
  } else {
    iters[sid] += 1;
    const double prev = rel[sid];
    rel_prev[sid] = prev;
    rel[sid] = relres;
    if (relres <= tol || relres > 0.5 * prev || !(relres == relres)) done[sid] = 1;
  }
}

cudaError_t launch_residual(const SysDev* sys, const int* list, int nsys, const int32_t* rowptr,
                            const int32_t* colidx, const double* vals, const double* b, const double* x,
                            double* r, double* rel, double* rel_prev, int* done, int* iters, double* partial,
                            int* ticket, double tol, int first, cudaStream_t st, const int* skip) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  residual_kernel<<<dim3(RES_CHUNKS, nsys), 256, 0, st>>>(sys, list, rowptr, colidx, vals, b, x, r, rel, rel_prev,
                                                          done, iters, partial, ticket, tol, first, skip);
  return cudaGetLastError();
}

#endif  // TPNS_BAND_PART == 1

#define TPNS_INST(T)                                                                                       \
  template cudaError_t launch_band_fill<T>(const SysDev*, const int*, int, const int32_t*, const int32_t*,  \
                                           const double*, T*, int, int64_t, cudaStream_t, const int*);      \
  template cudaError_t launch_band_lu<T>(const SysDev*, const int*, int, int, T*, T*, T*, T*, int*, int, int*,\
                                         int*, cudaStream_t, const int*, int, int);                                   \
  template cudaError_t launch_band_dinv<T>(const SysDev*, const int*, int, int, const T*, T*, cudaStream_t, \
                                           const int*);                                                     \
  template cudaError_t launch_band_to_slab<T>(const SysDev*, const int*, int, const T*, T*, T*,             \
                                              cudaStream_t);                                                \
  template cudaError_t launch_band_chol<T>(const SysDev*, const int*, int, T*, int*, cudaStream_t);         \
  template cudaError_t launch_chol_to_lu<T>(const SysDev*, const SysDev*, const int*, int, const T*, T*,    \
                                            cudaStream_t);                                                  \
  template cudaError_t launch_band_solve<T>(const SysDev*, const int*, int, int, int, const T*, const T*,   \
                                            const T*, const double*, double*, int, const int*, int*,        \
                                            cudaStream_t, const int*, T*);                                  \
  template bool band_solve_fits_smem<T>(int, int);                                                          \
  template size_t band_lu_smem_bytes<T>(int);
// this file is compiled once per element type (kernels_band_f32.cu, kernels_band_f64.cu)
#if TPNS_BAND_PART == 1
TPNS_INST(float)
#elif TPNS_BAND_PART == 2
TPNS_INST(double)
#else
#error "compile kernels_band_f32.cu or kernels_band_f64.cu"
#endif

}  // namespace tpns
