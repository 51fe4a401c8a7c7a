// Multifrontal LU and triangular solves of the local Oseen systems (Algorithm 3 Step 3(2),
// eq. uclocalFully), scheduled as a dataflow over the elimination trees of all systems.
//
// One persistent launch factors every front of every system.  The fronts are numbered in a
// topological order (children first) that puts the fronts with the longest estimated
// remaining chain to their root first; each CTA takes the next front from an atomic counter,
// waits until the front's children are finished (a flag per front, tagged with the
// launch's epoch, bounded wait) and factors the whole front itself.  A CTA only waits for
// fronts that CTAs which started before it have taken, so no launch geometry or
// co-residency is needed for progress, and a parent starts as soon as its own children
// are done (no level barriers).  Per front (dense, column-major, unpivoted):
//   assembly   every column: zero, the CSR values the front owns, then the Schur
//              complements of the children added column by column (extend-add), one warp
//              per column, children in a fixed order: no atomics, deterministic;
//   panel k    warp 0 factors the 32 x 32 pivot block (pivot rows broadcast by shuffles),
//              then all threads form L21 = A21 U11^{-1} and U12 = L11^{-1} A12 in place by
//              substitution (the inverses of the blocks' triangles, which only the solves
//              use, are formed afterwards for all blocks at once);
//   update k   A22 -= L21 U12.  FP32 fronts: 128 x 128 chunks; the threads write both
//              operands into shared memory as core-matrix tiles with every value split into
//              two TF32 parts, one thread issues tcgen05.mma kind::tf32 (hi*hi + hi*lo +
//              lo*hi, FP32 accumulation: the error-compensated split of Ootomo and Yokota,
//              2022, which keeps the product close to FP32 accuracy) into a 128 x 128
//              tensor-memory accumulator, and all warps read it back with tcgen05.ld and
//              subtract it from the front.  FP64 fronts (and FP32 fronts on request) use a
//              CUDA-core tile product.
// The Schur complement left in a front's trailing block is consumed by its parent.
//
// Large fronts (order >= a threshold, and their ancestors) are left out of that launch and
// factored afterwards by all CTAs together, one tree level at a time: flat assembly passes,
// then per pivot block a panel launch and a tile-parallel update launch (the trailing
// updates of every four pivot blocks grouped, the Schur block updated once with all pivot
// columns).
//
// Solves (one pass of iterative refinement), one launch with the same scheduling: the
// forward tasks in that order (a front waits for its children: right-hand side plus the
// children's update vectors, the pivot blocks through the inverses of L11's diagonal
// blocks, then the L columns below), then the backward tasks in reverse order (a front
// waits for its own forward task and its parent: U12 against the ancestors' correction,
// then the inverses of U11's diagonal blocks), adding the correction to x.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "kernels.hpp"
#include "mf.hpp"

namespace tpns {
namespace {

constexpr int MF_THREADS = 256;           // factorisation CTA
constexpr int MF_STHREADS = 128;          // solve CTA: fronts are small, more of them in flight per SM
constexpr int MF_SOLVE_WIDE_M = 1024;     // solves with fronts of at least this order use 512-thread CTAs
constexpr int MF_WAIT_LIMIT = 1 << 22;
constexpr int MF_CN = MF_TILE;             // columns of one tensor-core update chunk (rows: MF_TILE)
constexpr int MF_TMEM_COLS = MF_CN;        // one 128 x 128 FP32 accumulator
constexpr int MF_SMEM = 226 * 1024;        // dynamic shared memory of the factorisation (near the opt-in maximum)
constexpr int DS = MF_NB + 1;              // padded stride of the 32 x 32 shared tiles
constexpr int DSV = MF_NB + 4;             // row stride of the pivot block in shared memory (16-byte rows)

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false if the limit was reached
__device__ __forceinline__ bool mb_wait(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < MF_WAIT_LIMIT; ++it)
    if (mb_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// bounded wait for a flag to reach value v; false if the limit was reached
__device__ __forceinline__ bool wait_flag(const int* p, int v) {
  for (int it = 0; ld_acquire(p) != v; ++it) {
    if (it > MF_WAIT_LIMIT) return false;
    __nanosleep(32);
  }
  return true;
}

// tensor memory and the fifth-generation tensor core
__device__ __forceinline__ void tm_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma_tf32(uint32_t dtm, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns of tensor memory, one lane per thread (the
// registers are valid after tm_wait_ld)
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major: 8-row x 16-byte core matrices;
// lbo = byte distance of core matrices along K, sbo = along M/N (8-row groups).
__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128.
constexpr uint32_t MF_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(MF_CN >> 3) << 17) |
                              ((uint32_t)(MF_TILE >> 4) << 24);

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// Loads of data written by other CTAs in the same launch (a child's Schur complement, the
// solves' vectors) bypass L1; a front's own entries, written and read by one CTA (in global
// or in shared memory), use plain loads.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}
// offset (elements) of (row, k) in packed rows x 32 operand tiles: core matrices of 8 rows
// x 4 values; the K-chunks of a row group are adjacent (128 bytes apart), row groups follow
// each other (1024 bytes apart)
__device__ __forceinline__ int pack_idx(int r, int k) { return ((r >> 3) * 8 + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }
__device__ __forceinline__ bool bad_val(float v) { return !(fabsf(v) > 0.0f) || !(fabsf(v) < INFINITY); }
__device__ __forceinline__ bool bad_val(double v) { return !(fabs(v) > 0.0) || !(fabs(v) < (double)INFINITY); }

// The phases of a front are separate (not inlined) device functions: each then keeps its
// register arrays in registers instead of sharing one allocation with every other phase.

// ---------------------------------------------------------------- pivot block
__device__ __forceinline__ float shfl_t(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_t(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <typename T>
struct alignas(16) PanelSmem {
  T D[MF_NB][DSV];     // the pivot block's LU (unit L below, U on and above the diagonal)
  T R[MF_NB];          // reciprocals of the pivots
  T P[MF_NB];          // the pivot row being broadcast
};

// Factor the pivot block of rows / columns k0 .. k0 + kb - 1 (padded to 32 with the
// identity) in place: S.D holds unit L below and U on and above the diagonal, S.R the
// pivots' reciprocals.  All threads call; a zero or non-finite pivot sets bit 0 of *s_flag.
// Warp 0 holds one row per lane; at step k lane k publishes its (final) row in shared memory
// and the lanes below eliminate against it.  The inverses of the block's triangles, which
// only the solves need, are formed afterwards for all blocks at once (mf_dinv_kernel).
template <typename T>
__device__ __noinline__ void pivot_block(PanelSmem<T>& S, const T* __restrict__ F, int ld, int k0, int kb,
                                         int* s_flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    T a[MF_NB];   // lane i holds row i
    const T* row = F + (int64_t)k0 * ld + k0 + (lane < kb ? lane : 0);
#pragma unroll
    for (int c = 0; c < MF_NB; ++c) a[c] = row[(int64_t)(c < kb ? c : 0) * ld];
#pragma unroll
    for (int c = 0; c < MF_NB; ++c)
      if (c >= kb || lane >= kb) a[c] = (c == lane) ? T(1) : T(0);
    bool bad = false;
    // step k: lane k's (final) row is broadcast by shuffles; the lanes below eliminate
#pragma unroll
    for (int k = 0; k < MF_NB; ++k) {
      const T piv = shfl_t(a[k], k);
      if (k < kb) bad |= bad_val(piv);
      const T rp = recip(piv);
      if (lane == 0) S.R[k] = rp;
      const T l = a[k] * rp;
#pragma unroll
      for (int c = k + 1; c < MF_NB; ++c) {
        const T pc = shfl_t(a[c], k);
        if (lane > k) a[c] -= l * pc;
      }
      if (lane > k) a[k] = l;
    }
#pragma unroll
    for (int c = 0; c < MF_NB; ++c) S.D[lane][c] = a[c];
    if (lane == 0 && bad) atomicOr(s_flag, 1);
  }
  __syncthreads();
}

__device__ __forceinline__ void put_split(float* hi, float* lo, int l, const float (&o)[MF_NB]) {
#pragma unroll
  for (int c4 = 0; c4 < MF_NB; c4 += 4) {
    float4 h, q;
    h.x = tf32_rn(o[c4]); q.x = tf32_rn(o[c4] - h.x);
    h.y = tf32_rn(o[c4 + 1]); q.y = tf32_rn(o[c4 + 1] - h.y);
    h.z = tf32_rn(o[c4 + 2]); q.z = tf32_rn(o[c4 + 2] - h.z);
    h.w = tf32_rn(o[c4 + 3]); q.w = tf32_rn(o[c4 + 3] - h.w);
    *reinterpret_cast<float4*>(hi + pack_idx(l, c4)) = h;
    *reinterpret_cast<float4*>(lo + pack_idx(l, c4)) = q;
  }
}
__device__ __forceinline__ void put_split(float*, float*, int, const double (&)[MF_NB]) {}

// Four consecutive entries of a 16-byte-aligned row of the pivot block in shared memory (all
// threads of a warp read the same address: one broadcast vector load)
__device__ __forceinline__ void ld4(const float* p, float (&d)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&d)[4]) {
  const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
  d[0] = v0.x; d[1] = v0.y; d[2] = v1.x; d[3] = v1.y;
}

// L rows r in [k1, m): F[r, k0:k0+kb] <- F[r, k0:k0+kb] U11^{-1}; U columns c in [k1, m):
// F[k0:k0+kb, c] <- L11^{-1} F[k0:k0+kb, c], by substitution with the factored pivot block,
// which both read by rows (U's rows for the L rows, L's rows for the U columns), four entries
// at a time.  One thread per row or column.  With `pk`
// (FP32 tensor-core path) the first 128 rows and 256 columns also go straight into the
// packed operand tiles of the first update chunk.
// The rows / columns handled by a thread are q_first, q_first + q_step, ... (default: this
// CTA's threads over all of them).
template <typename T>
__device__ __noinline__ void panel_lu(const PanelSmem<T>& S, T* __restrict__ F, int ld, int m, int k0, int kb, int k1,
                                      float* pAh = nullptr, float* pAl = nullptr, float* pBh = nullptr,
                                      float* pBl = nullptr, int q_first = -1, int q_step = 0) {
  const int rest = m - k1;
  if (q_step == 0) {
    q_first = threadIdx.x;
    q_step = blockDim.x;
  }
  for (int q = q_first; q < 2 * rest; q += q_step) {
    const bool row = q < rest;
    const int idx = k1 + (row ? q : q - rest);
    T a[MF_NB];
    // every load from a valid address first (clamped), masked afterwards
    const T* base = row ? F + (int64_t)k0 * ld + idx : F + (int64_t)idx * ld + k0;
    const int64_t step = row ? ld : 1;
#pragma unroll
    for (int c = 0; c < MF_NB; ++c) a[c] = base[(c < kb ? c : 0) * step];
#pragma unroll
    for (int c = 0; c < MF_NB; ++c)
      if (c >= kb) a[c] = T(0);
    T o[MF_NB];
    if (row) {
      // l U11 = a: l_c = a_c / u_cc, then a_c' -= l_c u_cc' for c' > c (row c of U)
#pragma unroll
      for (int c = 0; c < MF_NB; ++c) {
        const T v = a[c] * S.R[c];
        o[c] = v;
#pragma unroll
        for (int c4 = (c + 1) & ~3; c4 < MF_NB; c4 += 4) {
          T d[4];
          ld4(&S.D[c][c4], d);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c4 + j > c) a[c4 + j] -= v * d[j];
        }
      }
    } else {
      // L11 u = a (unit diagonal): u_c = a_c - l_c0 u_0 - l_c1 u_1 - ... (row c of L; the
      // terms are taken in the order of the column-oriented elimination, so the rounding is
      // the same)
#pragma unroll
      for (int c = 0; c < MF_NB; ++c) {
        T acc = a[c];
#pragma unroll
        for (int c4 = 0; c4 < c; c4 += 4) {
          T d[4];
          ld4(&S.D[c][c4], d);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c4 + j < c) acc -= d[j] * o[c4 + j];
        }
        o[c] = acc;
      }
    }
    if (row) {
#pragma unroll
      for (int c2 = 0; c2 < MF_NB; ++c2)
        if (c2 < kb) F[(int64_t)(k0 + c2) * ld + idx] = o[c2];
      if (pAh && idx - k1 < MF_TILE) put_split(pAh, pAl, idx - k1, o);
    } else {
#pragma unroll
      for (int c2 = 0; c2 < MF_NB; ++c2)
        if (c2 < kb) F[(int64_t)idx * ld + k0 + c2] = o[c2];
      if (pBh && idx - k1 < MF_CN) put_split(pBh, pBl, idx - k1, o);
    }
  }
  __syncthreads();
}

// CUDA-core tile update: F[r0:r0+128, c0:c0+128] -= L21 U12 (K = kb), reading the panel
// from the front.  Thread (tx, ty) owns rows tx + 16 a and columns ty + 16 b.
// (rows below m, columns below cl: cl = m by default)
template <typename T>
__device__ __noinline__ void update_tile_fma(T* __restrict__ F, int ld, int m, int k0, int kb, int r0, int c0, T* As, T* Bs,
                                             int cl = -1) {
  if (cl < 0) cl = m;
  constexpr int W = MF_TILE + 4;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int u = 0; u < MF_NB * MF_TILE / MF_THREADS; ++u) {
    const int q = tid + u * MF_THREADS;
    const int k = q / MF_TILE, r = q % MF_TILE;
    As[k * W + r] = (k < kb && r0 + r < m) ? F[(int64_t)(k0 + k) * ld + r0 + r] : T(0);
    const int c = q / MF_NB, kk = q % MF_NB;
    Bs[kk * W + c] = (kk < kb && c0 + c < cl) ? F[(int64_t)(c0 + c) * ld + k0 + kk] : T(0);
  }
  __syncthreads();
  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
  for (int k = 0; k < kb; ++k) {
    T av[8], bv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) av[a] = As[k * W + tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 8; ++b) bv[b] = Bs[k * W + ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int c = c0 + ty + 16 * b;
    if (c >= cl) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = r0 + tx + 16 * a;
      if (r < m) {
        T* p = F + (int64_t)c * ld + r;
        *p = *p - acc[a][b];
      }
    }
  }
  __syncthreads();
}

// Shared memory of the FP32 tensor-core path: operand chunks (A = 128 rows of L21, B = 128
// columns of U12, 32 values each, TF32 hi and lo parts), the pivot block, barrier, TMEM
// address (69 KB); the rest of the CTA's shared memory holds the front when it fits.
struct TcSmem {
  float Ahi[MF_TILE * MF_NB], Alo[MF_TILE * MF_NB], Bhi[MF_CN * MF_NB], Blo[MF_CN * MF_NB];
  PanelSmem<float> P;
  uint64_t bar;
  uint32_t tmem;
};

// Pack rows (or columns) [l0, l0 + n) of the panel into core-matrix tiles, each value split
// into TF32 hi and lo parts: row: L21 rows r0 + l (values F[r, k0 + c]); column: U12 columns
// (values F[k0 + c, c0 + l]).  Entries past `valid` or kb are zero.
__device__ __forceinline__ void pack_panel(const float* __restrict__ F, int ld, int k0, int kb, int first, int valid,
                                           bool row, int l, float* hi, float* lo) {
  const bool ok = l < valid;
  const int li = ok ? l : 0;
  const float* base = row ? F + (int64_t)k0 * ld + first + li : F + (int64_t)(first + li) * ld + k0;
  const int64_t step = row ? ld : 1;
  float v[MF_NB];
#pragma unroll
  for (int c = 0; c < MF_NB; ++c) v[c] = base[(c < kb ? c : 0) * step];
#pragma unroll
  for (int c = 0; c < MF_NB; ++c)
    if (!ok || c >= kb) v[c] = 0.f;
#pragma unroll
  for (int c4 = 0; c4 < MF_NB; c4 += 4) {
    float4 h, o;
    h.x = tf32_rn(v[c4]); o.x = tf32_rn(v[c4] - h.x);
    h.y = tf32_rn(v[c4 + 1]); o.y = tf32_rn(v[c4 + 1] - h.y);
    h.z = tf32_rn(v[c4 + 2]); o.z = tf32_rn(v[c4 + 2] - h.z);
    h.w = tf32_rn(v[c4 + 3]); o.w = tf32_rn(v[c4 + 3] - h.w);
    *reinterpret_cast<float4*>(hi + pack_idx(l, c4)) = h;
    *reinterpret_cast<float4*>(lo + pack_idx(l, c4)) = o;
  }
}

// One thread: the twelve products of a chunk (four K-steps of 8, each hi*hi + hi*lo + lo*hi)
// into the accumulator at tensor-memory address `tmem`, then a commit of their completion to
// the mbarrier.
__device__ __noinline__ void issue_chunk(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo,
                                         uint32_t tmem, uint64_t* bar, bool accumulate = false) {
  const uint32_t ah = su32(Ahi), al = su32(Alo), bh = su32(Bhi), bl = su32(Blo);
#pragma unroll 1
  for (int kk = 0; kk < MF_NB / 8; ++kk) {
    const uint32_t o = kk * 256;   // 8 TF32 values = two 16-byte core matrices along K
    tc_mma_tf32(tmem, sm_desc(ah + o, 128, 1024), sm_desc(bh + o, 128, 1024), MF_IDESC, kk > 0 || accumulate);
    tc_mma_tf32(tmem, sm_desc(ah + o, 128, 1024), sm_desc(bl + o, 128, 1024), MF_IDESC, 1);
    tc_mma_tf32(tmem, sm_desc(al + o, 128, 1024), sm_desc(bh + o, 128, 1024), MF_IDESC, 1);
  }
  tc_commit(bar);
}

// Trailing update F[k1:m, k1:m] -= L21 U12 of one pivot block on the tensor cores, in
// chunks of 128 rows x 128 columns (one accumulator in tensor memory).
__device__ __noinline__ void update_tc(TcSmem& S, float* __restrict__ F, int ld, int m, int k0, int kb, int k1,
                                       unsigned& ph, int* s_flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c0 = k1; c0 < m; c0 += MF_CN) {
    const int nc = min(MF_CN, m - c0);
    for (int r0 = k1; r0 < m; r0 += MF_TILE) {
      const int nr = min(MF_TILE, m - r0);
      // operands: A rows once per chunk row, B columns once per chunk column; the panel
      // pass already packed those of the first chunk
      const bool first = r0 == k1 && c0 == k1;
      if (!first && tid < MF_TILE) pack_panel(F, ld, k0, kb, r0, nr, true, tid, S.Ahi, S.Alo);
      if (!first && r0 == k1 && tid < MF_CN) pack_panel(F, ld, k0, kb, c0, nc, false, tid, S.Bhi, S.Blo);
      // the tensor core reads shared memory through the async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_before();
      __syncthreads();
      tc_after();
      if (tid == 0) issue_chunk(S.Ahi, S.Alo, S.Bhi, S.Blo, S.tmem, &S.bar);
      if (!mb_wait(&S.bar, ph) && lane == 0) atomicOr(s_flag, 2);
      ph ^= 1u;
      tc_after();
      // epilogue: warp w reads accumulator lanes 32 (w % 4) .., columns 64 (w / 4) ..
      const int q4 = warp & 3, hcol = warp >> 2;
      const int r = r0 + 32 * q4 + lane;
      const int cb = c0 + 64 * hcol;
      if (r0 + 32 * q4 < m && cb < m) {   // warp-uniform
        const uint32_t base = S.tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(64 * hcol);
        const int rr = r < m ? r : m - 1;
#pragma unroll 1
        for (int h16 = 0; h16 < 4; ++h16) {
          const int cb2 = cb + 16 * h16;
          if (cb2 >= m) break;
          uint32_t d[16];
          tm_ld16(base + (uint32_t)(16 * h16), d);
          // the front's current values, all loads in flight together (clamped addresses)
          float f[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) f[c] = F[(int64_t)(cb2 + c < m ? cb2 + c : m - 1) * ld + rr];
          tm_wait_ld();
          if (r < m) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
              if (cb2 + c < m) F[(int64_t)(cb2 + c) * ld + r] = f[c] - __uint_as_float(d[c]);
          }
        }
      }
      tc_before();
      __syncthreads();
      tc_after();
    }
  }
}

// ---------------------------------------------------------------- factorisation
struct MFArgs {
  const MFSysDev* sys;
  const MFFrontDev* fronts;
  int task0, ntask;   // fronts task0 .. task0 + ntask - 1 are factored
  const int32_t* relmap;
  const int64_t* colptr;
  const int32_t* orig_k;
  const int32_t* orig_ij;   // row | column << 16 in the front
  const double* vals;
  int* status;
  int* sched;   // [0] task counter, [1] finished CTAs, [2] epoch
  int* flag;    // per front: epoch when factored
};

// Assemble a front in three passes over all of its entries, separated by barriers: zero,
// the CSR values it owns (distinct positions), then the Schur complement of each child in
// turn (distinct positions within one child), so the sums do not depend on scheduling.
template <typename T>
__device__ __noinline__ void assemble_front(const MFArgs& A, const MFFrontDev& Fd, T* __restrict__ F, int ld,
                                           const T* __restrict__ Fall, const double* vals) {
  const int tid = threadIdx.x;
  const int m = Fd.m;
  for (int q = tid; q < ld * m; q += MF_THREADS) F[q] = T(0);
  __syncthreads();
  {
    const int64_t b = A.colptr[Fd.colptr_off], e = A.colptr[Fd.colptr_off + m];
    for (int64_t q0 = b + tid; q0 < e; q0 += 4 * MF_THREADS) {
      int32_t ij[4];
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t q = q0 + (int64_t)u * MF_THREADS;
        ij[u] = q < e ? A.orig_ij[q] : -1;
        v[u] = q < e ? vals[A.orig_k[q]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ij[u] >= 0) F[(int64_t)(ij[u] >> 16) * ld + (ij[u] & 0xFFFF)] = (T)v[u];
    }
  }
  __syncthreads();
  for (int c = 0; c < Fd.nchild; ++c) {
    const MFFrontDev& C = A.fronts[c == 0 ? Fd.child0 : Fd.child1];
    const int qc = C.m - C.p;
    const T* src = Fall + C.f_off + (int64_t)C.p * C.ld + C.p;
    const int32_t* rm = A.relmap + C.relmap_off;
    const int tot = qc * qc;
    for (int q0 = tid; q0 < tot; q0 += 4 * MF_THREADS) {
      T v[4];
      int dst[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * MF_THREADS;
        dst[u] = -1;
        v[u] = T(0);
        if (q < tot) {
          const int ic = q % qc, jc = q / qc;
          v[u] = ldcg(src + (int64_t)jc * C.ld + ic);
          dst[u] = rm[jc] * ld + rm[ic];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) F[dst[u]] += v[u];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int next_task(int* sched, int* s_task) {
  __syncthreads();
  if (threadIdx.x == 0) *s_task = atomicAdd(&sched[0], 1);
  __syncthreads();
  return *s_task;
}

// the last CTA to finish resets the task counter and advances the epoch for the next launch
__device__ __forceinline__ void finish_launch(int* sched) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
      atomicExch(&sched[0], 0);
      atomicExch(&sched[1], 0);
      __threadfence();
      atomicAdd(&sched[2], 1);
    }
  }
}

template <typename T, bool TC>
__global__ void __launch_bounds__(MF_THREADS, 1)
    mf_factor_kernel(MFArgs A, T* __restrict__ Fall, T* __restrict__ dinv) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int s_task, s_flag;
  const int tid = threadIdx.x;
  TcSmem& TS = *reinterpret_cast<TcSmem*>(smem_raw);
  PanelSmem<T>* Pp;
  T* As = nullptr;
  if constexpr (TC) {
    Pp = reinterpret_cast<PanelSmem<T>*>(&TS.P);
  } else {
    As = reinterpret_cast<T*>(smem_raw);
    Pp = reinterpret_cast<PanelSmem<T>*>(smem_raw + (size_t)2 * MF_NB * (MF_TILE + 4) * sizeof(T));
  }
  PanelSmem<T>& P = *Pp;
  // the front itself goes to the shared memory left after the fixed part when it fits
  constexpr size_t fixed = TC ? sizeof(TcSmem) : (size_t)2 * MF_NB * (MF_TILE + 4) * sizeof(T) + sizeof(PanelSmem<T>);
  constexpr size_t fs_off = (fixed + 127) & ~(size_t)127;
  T* Fs = reinterpret_cast<T*>(smem_raw + fs_off);
  const int64_t fs_cap = (int64_t)(MF_SMEM - fs_off) / (int64_t)sizeof(T);
  const int epoch = ld_acquire(&A.sched[2]);
  unsigned ph = 0;
  if constexpr (TC) {
    if (tid == 0) {
      mb_init(&TS.bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) tm_alloc(&TS.tmem, MF_TMEM_COLS);
    tc_before();
    __syncthreads();
    tc_after();
  }
  for (;;) {
    const int t = next_task(A.sched, &s_task);
    if (t >= A.ntask) break;
    const int f = A.task0 + t;
    const MFFrontDev& Fd = A.fronts[f];
    const MFSysDev& S = A.sys[Fd.sys];
    if (tid == 0) {
      s_flag = 0;
      if (Fd.nchild > 0 && !wait_flag(&A.flag[Fd.child0], epoch)) s_flag |= 4;
      if (Fd.nchild > 1 && !wait_flag(&A.flag[Fd.child1], epoch)) s_flag |= 4;
    }
    __syncthreads();
    T* Fg = Fall + Fd.f_off;
    const int lds = Fd.m | 1;   // odd stride: row-wise accesses in shared memory are conflict free
    const bool sh = (int64_t)Fd.m * lds <= fs_cap;
    T* F = sh ? Fs : Fg;
    const int ld = sh ? lds : Fd.ld;
    assemble_front<T>(A, Fd, F, ld, Fall, A.vals + S.val_off);
    for (int k0 = 0, kk = 0; k0 < Fd.p; k0 += MF_NB, ++kk) {
      const int kb = min(MF_NB, Fd.p - k0), k1 = k0 + kb;
      pivot_block<T>(P, F, ld, k0, kb, &s_flag);
      // the factored pivot block (row-major) for mf_dinv_kernel
      T* dv = dinv + Fd.dinv_off + (int64_t)kk * 2 * MF_NB * MF_NB + MF_NB * MF_NB;
      for (int q = tid; q < MF_NB * MF_NB; q += blockDim.x) dv[q] = P.D[q >> 5][q & 31];
      if (k1 >= Fd.m) {
        __syncthreads();
        continue;
      }
      if constexpr (TC) panel_lu<T>(P, F, ld, Fd.m, k0, kb, k1, TS.Ahi, TS.Alo, TS.Bhi, TS.Blo);
      else panel_lu<T>(P, F, ld, Fd.m, k0, kb, k1);
      if constexpr (TC) {
        if (s_flag & 2) continue;   // a bounded wait gave up: issue no further products
        update_tc(TS, F, ld, Fd.m, k0, kb, k1, ph, &s_flag);
      } else {
        const int nt = (Fd.m - k1 + MF_TILE - 1) / MF_TILE;
        for (int t = 0; t < nt * nt; ++t)
          update_tile_fma<T>(F, ld, Fd.m, k0, kb, k1 + (t % nt) * MF_TILE, k1 + (t / nt) * MF_TILE, As,
                             As + MF_NB * (MF_TILE + 4));
      }
    }
    __syncthreads();
    if (sh) {
      // factors and Schur complement to the front's place in global memory
      const int m = Fd.m;
      for (int q = tid; q < m * m; q += MF_THREADS) {
        const int j = q / m, i = q - j * m;
        Fg[(int64_t)j * Fd.ld + i] = Fs[j * lds + i];
      }
      __syncthreads();
    }
    if (tid == 0) {
      if (s_flag) atomicOr(&A.status[S.sid], s_flag);
      __threadfence();
      st_release(&A.flag[f], epoch);
    }
  }
  if constexpr (TC) {
    tc_before();
    __syncthreads();
    tc_after();
    if ((tid >> 5) == 0) tm_dealloc(TS.tmem, MF_TMEM_COLS);
  }
  finish_launch(A.sched);
}

// ---------------------------------------------------------------- large fronts
// Fronts of large order (and all their ancestors) are factored by many CTAs together,
// level by level of the elimination trees (all fronts of one height at once): a column-
// parallel assembly, then per 32-column pivot block one launch for the panel (every CTA of a
// front factors the 32 x 32 pivot block itself and substitutes its share of the L21 rows and
// U12 columns) and one launch for the trailing update, whose 128 x 128 tiles over all fronts
// of the level are spread over all CTAs (tensor cores for FP32 fronts, CUDA cores otherwise).
// Launch order on the stream orders the steps: no CTA waits for another.
struct MFBigArgs {
  const MFSysDev* sys;
  const MFFrontDev* fronts;
  const int32_t* list;   // fronts of this launch
  int nlist;
  const int32_t* relmap;
  const int64_t* colptr;
  const int32_t* orig_k;
  const int32_t* orig_ij;
  const double* vals;
  int* status;
};

// phase 0: zero the front; phase 3: place its CSR values (distinct positions); phase 1 / 2:
// add the Schur complement of child 0 / 1 (distinct positions within one child).  Each pass
// is a flat loop over the front's entries spread over the CTAs of the front (blockIdx.y).
template <typename T>
__global__ void __launch_bounds__(MF_THREADS) mf_big_assemble_kernel(MFBigArgs A, T* __restrict__ Fall, int phase) {
  const MFFrontDev& Fd = A.fronts[A.list[blockIdx.y]];
  T* F = Fall + Fd.f_off;
  const int ld = Fd.ld, m = Fd.m;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
  if (phase == 0) {
    const int64_t n = (int64_t)ld * m;
    for (int64_t q = first; q < n; q += step) F[q] = T(0);
    return;
  }
  if (phase == 3) {
    const double* vals = A.vals + A.sys[Fd.sys].val_off;
    const int64_t b = A.colptr[Fd.colptr_off], e = A.colptr[Fd.colptr_off + m];
    for (int64_t q = b + first; q < e; q += step) {
      const int32_t ij = A.orig_ij[q];
      F[(int64_t)(ij >> 16) * ld + (ij & 0xFFFF)] = (T)vals[A.orig_k[q]];
    }
    return;
  }
  if (phase > Fd.nchild) return;
  const MFFrontDev& C = A.fronts[phase == 1 ? Fd.child0 : Fd.child1];
  const int qc = C.m - C.p;
  const T* src = Fall + C.f_off + (int64_t)C.p * C.ld + C.p;
  const int32_t* rm = A.relmap + C.relmap_off;
  const int64_t n = (int64_t)qc * qc;
  for (int64_t q = first; q < n; q += step) {
    const int jc = (int)(q / qc), ic = (int)(q - (int64_t)jc * qc);
    F[(int64_t)rm[jc] * ld + rm[ic]] += ldcg(src + (int64_t)jc * C.ld + ic);
  }
}

// pivot block k0 of every listed front with p > k0: its LU (written by CTA 0 to the block's
// slot for mf_dinv_kernel) and the substitutions of L21 rows / U12 columns, spread over the
// CTAs of the front
template <typename T>
__global__ void __launch_bounds__(MF_THREADS, 2) mf_big_panel_kernel(MFBigArgs A, T* __restrict__ Fall,
                                                                  T* __restrict__ dinv, int k0) {
  __shared__ PanelSmem<T> P;
  __shared__ int s_flag;
  const MFFrontDev& Fd = A.fronts[A.list[blockIdx.y]];
  if (k0 >= Fd.p) return;
  if (threadIdx.x == 0) s_flag = 0;
  __syncthreads();
  T* F = Fall + Fd.f_off;
  const int ld = Fd.ld;
  const int kb = min(MF_NB, Fd.p - k0), k1 = k0 + kb;
  pivot_block<T>(P, F, ld, k0, kb, &s_flag);
  if (blockIdx.x == 0) {
    T* dv = dinv + Fd.dinv_off + (int64_t)(k0 / MF_NB) * 2 * MF_NB * MF_NB + MF_NB * MF_NB;
    for (int q = threadIdx.x; q < MF_NB * MF_NB; q += blockDim.x) dv[q] = P.D[q >> 5][q & 31];
    if (threadIdx.x == 0 && s_flag) atomicOr(&A.status[A.sys[Fd.sys].sid], s_flag);
  }
  if (k1 < Fd.m)
    panel_lu<T>(P, F, ld, Fd.m, k0, kb, k1, nullptr, nullptr, nullptr, nullptr,
                blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Trailing updates of the listed fronts, in 128 x 128 tiles taken round robin by the CTAs.
// The pivot columns [0, p) go in groups of MF_BIG_GROUP (a group [gs, ge), ge = min(gs +
// MF_BIG_GROUP, p)); for entries outside the Schur block the updates of a group are applied
// together once the group is factored, so that the trailing region is rewritten once per
// group instead of once per pivot block:
//   mode 1, pivot block k0 of group [gs, ge) (K = its 32 columns, k1 = k0 + 32): only the
//     group's own panels, rows [k1, m) x columns [k1, ge) and rows [k1, ge) x columns [ge, m);
//   mode 3, after the last pivot block of group [gs, ge) (K = the group's columns): the
//     entries the later pivot blocks need, rows [ge, m) x columns [ge, p) and rows [ge, p) x
//     columns [p, m);
//   mode 2, after the last pivot block (K = p): the Schur block [p, m) x [p, m) once (the
//     products of all pivot blocks accumulate in tensor memory, or in registers on the
//     CUDA-core path).
// Every entry thus receives the product of each earlier pivot block exactly once before it is
// read by a panel (the blocked right-looking LU with a two-level panel).
constexpr int MF_BIG_GROUP = 4 * MF_NB;
struct BigTile {
  int r0, c0, rl, cl;   // tile origin, row / column limits
};
__device__ __forceinline__ int ceil_tiles(int n) { return n > 0 ? (n + MF_TILE - 1) / MF_TILE : 0; }
// K range [kc0, kc1) of the products of a tile
__device__ __forceinline__ void big_krange(const MFFrontDev& Fd, int mode, int k0, int& kc0, int& kc1) {
  if (mode == 2) {
    kc0 = 0;
    kc1 = Fd.p;
  } else if (mode == 1) {
    kc0 = k0;
    kc1 = min(k0 + MF_NB, Fd.p);
  } else {
    kc0 = (k0 / MF_BIG_GROUP) * MF_BIG_GROUP;
    kc1 = min(kc0 + MF_BIG_GROUP, Fd.p);
  }
}
__device__ __forceinline__ int big_tiles(const MFFrontDev& Fd, int mode, int k0) {
  const int p = Fd.p, m = Fd.m;
  if (mode == 2) return m > p ? ceil_tiles(m - p) * ceil_tiles(m - p) : 0;
  if (k0 >= p) return 0;
  const int ge = min((k0 / MF_BIG_GROUP) * MF_BIG_GROUP + MF_BIG_GROUP, p);
  if (mode == 1) {
    const int k1 = min(k0 + MF_NB, p);
    if (k1 >= ge) return 0;
    return ceil_tiles(m - k1) + ceil_tiles(m - ge);   // ge - k1 < MF_TILE: one tile column / row
  }
  if (ge >= p) return 0;
  const int b = ceil_tiles(p - ge);
  return ceil_tiles(m - ge) * b + b * ceil_tiles(m - p);
}
__device__ __forceinline__ BigTile big_tile(const MFFrontDev& Fd, int mode, int k0, int tl) {
  const int p = Fd.p, m = Fd.m;
  BigTile T;
  if (mode == 2) {
    const int nt = ceil_tiles(m - p);
    T.r0 = p + (tl % nt) * MF_TILE; T.c0 = p + (tl / nt) * MF_TILE; T.rl = m; T.cl = m;
    return T;
  }
  const int ge = min((k0 / MF_BIG_GROUP) * MF_BIG_GROUP + MF_BIG_GROUP, p);
  if (mode == 1) {
    const int k1 = min(k0 + MF_NB, p);
    const int a = ceil_tiles(m - k1);
    if (tl < a) {
      T.r0 = k1 + tl * MF_TILE; T.c0 = k1; T.rl = m; T.cl = ge;
    } else {
      T.r0 = k1; T.c0 = ge + (tl - a) * MF_TILE; T.rl = ge; T.cl = m;
    }
    return T;
  }
  const int a = ceil_tiles(m - ge), b = ceil_tiles(p - ge);
  if (tl < a * b) {
    T.r0 = ge + (tl % a) * MF_TILE; T.c0 = ge + (tl / a) * MF_TILE; T.rl = m; T.cl = p;
  } else {
    tl -= a * b;
    T.r0 = ge + (tl % b) * MF_TILE; T.c0 = p + (tl / b) * MF_TILE; T.rl = p; T.cl = m;
  }
  return T;
}

// Operands of one K chunk (32 columns) of a 128 x 128 tile in the packed layout of pack_idx:
// L21 rows (A) and U12 columns (B), each split into TF32 hi and lo parts (64 KB).
struct TcOps {
  float Ahi[MF_TILE * MF_NB], Alo[MF_TILE * MF_NB], Bhi[MF_CN * MF_NB], Blo[MF_CN * MF_NB];
};
// Shared memory of the tensor-core trailing update: two operand stages, so that the next
// chunk is packed while the tensor core multiplies the current one, their mbarriers (each
// receives the commits of the chunks packed into its stage) and the accumulator's address.
struct BigUSmem {
  TcOps op[2];
  uint64_t bar[2];
  uint32_t tmem;
};

// A tile of the update with the K range of its products (one chunk per pivot block)
struct UTile {
  float* F;
  int ld, r0, c0, rl, cl, kc0, kc1;
};
__device__ __forceinline__ UTile u_tile(const MFBigArgs& A, float* Fall, const int* s_pre, int mode, int k0, int t,
                                        int& fi) {
  while (s_pre[fi + 1] <= t) ++fi;
  const MFFrontDev& Fd = A.fronts[A.list[fi]];
  const BigTile G = big_tile(Fd, mode, k0, t - s_pre[fi]);
  UTile u;
  u.F = Fall + Fd.f_off;
  u.ld = Fd.ld;
  u.r0 = G.r0; u.c0 = G.c0; u.rl = G.rl; u.cl = G.cl;
  big_krange(Fd, mode, k0, u.kc0, u.kc1);
  return u;
}

// Half of one operand row or column of chunk kc (16 of its 32 values, columns kc + 16 h ..):
// A (op 0): L21 row r0 + l, values F[kc + c, r0 + l]; B (op 1): U12 column c0 + l, values
// F[c0 + l, kc + c].  Loads only (clamped addresses, masked afterwards), so that they stay in
// flight while the tensor core works; entries past the tile or the pivot range are zero.
__device__ __forceinline__ void load_half(const UTile& u, int kc, int op, int l, int h, float (&v)[16]) {
  const int kb = min(MF_NB, u.kc1 - kc);
  const int first = op == 0 ? u.r0 : u.c0;
  const int valid = op == 0 ? u.rl - u.r0 : u.cl - u.c0;
  const bool ok = l < valid;
  const int li = ok ? l : 0;
  const float* base = op == 0 ? u.F + (int64_t)kc * u.ld + first + li : u.F + (int64_t)(first + li) * u.ld + kc;
  const int64_t step = op == 0 ? u.ld : 1;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int cc = 16 * h + c;
    v[c] = base[(cc < kb ? cc : 0) * step];
  }
#pragma unroll
  for (int c = 0; c < 16; ++c)
    if (!ok || 16 * h + c >= kb) v[c] = 0.f;
}
__device__ __forceinline__ void store_half(TcOps& O, int op, int l, int h, const float (&v)[16]) {
  float* hi = op == 0 ? O.Ahi : O.Bhi;
  float* lo = op == 0 ? O.Alo : O.Blo;
#pragma unroll
  for (int c4 = 0; c4 < 16; c4 += 4) {
    float4 a, b;
    a.x = tf32_rn(v[c4]); b.x = tf32_rn(v[c4] - a.x);
    a.y = tf32_rn(v[c4 + 1]); b.y = tf32_rn(v[c4 + 1] - a.y);
    a.z = tf32_rn(v[c4 + 2]); b.z = tf32_rn(v[c4 + 2] - a.z);
    a.w = tf32_rn(v[c4 + 3]); b.w = tf32_rn(v[c4 + 3] - a.w);
    *reinterpret_cast<float4*>(hi + pack_idx(l, 16 * h + c4)) = a;
    *reinterpret_cast<float4*>(lo + pack_idx(l, 16 * h + c4)) = b;
  }
}

// The tensor-core update of this CTA's tiles (t = blockIdx.x, + gridDim.x, ...), as one
// sequence of K chunks: chunk g is packed into stage g % 2 once the products of chunk g - 2
// (the stage's previous contents) have completed, one thread issues its products, and the
// loads of chunk g + 1 are in flight while they run.  After a tile's last chunk, the epilogue
// waits for its products and subtracts the accumulator from the tile (warp w: accumulator
// lanes 32 (w % 4) .., columns 32 (w / 4) ..); the tile's current values were loaded while its
// first products ran.  512 threads: thread (op, h, l) packs half of L21 row l (op 0) or of U12
// column l (op 1).  Every wait is bounded; a wait that gives up stops the sequence (a uniform
// decision) and sets bit 1 of the system's status.
__device__ __forceinline__ void big_update_tc(const MFBigArgs& A, float* Fall, const int* s_pre, int k0, int mode) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  BigUSmem& S = *reinterpret_cast<BigUSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int op = tid >> 8, h = (tid >> 7) & 1, l = tid & (MF_TILE - 1);
  const int q4 = warp & 3, hcol = warp >> 2;
  if (tid == 0) {
    mb_init(&S.bar[0], 1);
    mb_init(&S.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tm_alloc(&S.tmem, MF_TMEM_COLS);
  tc_before();
  __syncthreads();
  tc_after();
  const int total = s_pre[A.nlist];
  int t = blockIdx.x, fi = 0, issued = 0;
  bool stopped = false;
  if (t < total) {
    UTile cur = u_tile(A, Fall, s_pre, mode, k0, t, fi);
    int kc = cur.kc0;
    float v[16], f[32];
    load_half(cur, kc, op, l, h, v);
    for (;;) {
      const int g = issued, s = g & 1;
      // the stage's previous chunk (g - 2) has been multiplied
      const bool free_ok = g < 2 || mb_wait(&S.bar[s], ((g - 2) >> 1) & 1);
      store_half(S.op[s], op, l, h, v);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_before();
      stopped = __syncthreads_or(!free_ok);
      tc_after();
      if (stopped) break;
      const bool first = kc == cur.kc0, last = kc + MF_NB >= cur.kc1;
      if (tid == 0) issue_chunk(S.op[s].Ahi, S.op[s].Alo, S.op[s].Bhi, S.op[s].Blo, S.tmem, &S.bar[s], !first);
      ++issued;
      const int r = cur.r0 + 32 * q4 + lane, cb = cur.c0 + 32 * hcol;
      const int rr = r < cur.rl ? r : cur.rl - 1;
      if (first) {
#pragma unroll
        for (int c = 0; c < 32; ++c) f[c] = cur.F[(int64_t)(cb + c < cur.cl ? cb + c : cur.cl - 1) * cur.ld + rr];
      }
      // the next chunk: the tile's next 32 pivot columns, or the first chunk of the next tile
      UTile nxt = cur;
      int nkc = kc + MF_NB;
      bool more = true;
      if (last) {
        t += gridDim.x;
        more = t < total;
        if (more) {
          nxt = u_tile(A, Fall, s_pre, mode, k0, t, fi);
          nkc = nxt.kc0;
        }
      }
      if (more) load_half(nxt, nkc, op, l, h, v);
      if (last) {
        const bool ok = mb_wait(&S.bar[s], (g >> 1) & 1);
        tc_after();
        if (cur.r0 + 32 * q4 < cur.rl && cb < cur.cl) {   // warp-uniform
          const uint32_t base = S.tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(32 * hcol);
#pragma unroll
          for (int h16 = 0; h16 < 2; ++h16) {
            const int cb2 = cb + 16 * h16;
            uint32_t d[16];
            tm_ld16(base + (uint32_t)(16 * h16), d);
            tm_wait_ld();
            if (r < cur.rl) {
#pragma unroll
              for (int c = 0; c < 16; ++c)
                if (cb2 + c < cur.cl) cur.F[(int64_t)(cb2 + c) * cur.ld + r] = f[16 * h16 + c] - __uint_as_float(d[c]);
            }
          }
        }
        // the accumulator is free for the next tile
        tc_before();
        stopped = __syncthreads_or(!ok);
        tc_after();
        if (stopped) break;
      }
      if (!more) break;
      cur = nxt;
      kc = nkc;
    }
  }
  // products still in flight (only after a wait gave up) complete before the accumulator is
  // released
  if (issued > 0 && !mb_wait(&S.bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1)) stopped = true;
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0) tm_dealloc(S.tmem, MF_TMEM_COLS);
  if (tid == 0 && stopped) atomicOr(&A.status[A.sys[A.fronts[A.list[0]].sys].sid], 2);
}

// Tensor-core variant (FP32 fronts): big_update_tc, 512 threads; CUDA-core variant: MF_THREADS
// (the 16 x 16 thread layout of update_tile_fma), one tile after another.
constexpr int MF_BIG_UTHREADS = 512;
template <typename T, bool TC>
__global__ void __launch_bounds__(TC ? MF_BIG_UTHREADS : MF_THREADS, 1)
    mf_big_update_kernel(MFBigArgs A, T* __restrict__ Fall, int k0, int mode) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int s_pre[MF_BIG_LIST + 1];
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < A.nlist; ++i) {
      s_pre[i] = acc;
      acc += big_tiles(A.fronts[A.list[i]], mode, k0);
    }
    s_pre[A.nlist] = acc;
  }
  __syncthreads();
  if constexpr (TC) {
    big_update_tc(A, reinterpret_cast<float*>(Fall), s_pre, k0, mode);
  } else {
    const int total = s_pre[A.nlist];
    int fi = 0;
    T* As = reinterpret_cast<T*>(smem_raw);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      while (s_pre[fi + 1] <= t) ++fi;
      const MFFrontDev& Fd = A.fronts[A.list[fi]];
      const BigTile G = big_tile(Fd, mode, k0, t - s_pre[fi]);
      int kc0, kc1;
      big_krange(Fd, mode, k0, kc0, kc1);
      for (int kc = kc0; kc < kc1; kc += MF_NB)
        update_tile_fma<T>(Fall + Fd.f_off, Fd.ld, G.rl, kc, min(MF_NB, kc1 - kc), G.r0, G.c0, As,
                           As + MF_NB * (MF_TILE + 4), G.cl);
    }
  }
}

// ---------------------------------------------------------------- block inverses
// For every pivot block in the list (offset of its 2 x 32 x 32 slot): read the factored block
// (row-major, second half of the slot), write L11^{-1} (unit lower) to the first half and
// U11^{-1} to the second.  One warp per block, lane j forms column j of each inverse.
template <typename T>
__global__ void __launch_bounds__(256) mf_dinv_kernel(T* __restrict__ dinv, const int64_t* __restrict__ blocks, int nblk) {
  __shared__ T B[8][MF_NB][DS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * 8 + w;
  if (b >= nblk) return;
  T* slot = dinv + blocks[b];
  T(&D)[MF_NB][DS] = B[w];
#pragma unroll
  for (int i = 0; i < MF_NB; ++i) D[i][lane] = slot[MF_NB * MF_NB + i * MF_NB + lane];
  __syncwarp();
  T u[MF_NB], l[MF_NB];
#pragma unroll
  for (int i = 0; i < MF_NB; ++i) {
    u[i] = (i == lane) ? T(1) : T(0);
    l[i] = u[i];
  }
  // U^{-1} e_lane, right-looking back substitution
#pragma unroll
  for (int i = MF_NB - 1; i >= 0; --i) {
    u[i] = u[i] / D[i][i];
#pragma unroll
    for (int k = 0; k < i; ++k) u[k] -= D[k][i] * u[i];
  }
  // L^{-1} e_lane (unit diagonal), right-looking forward substitution
#pragma unroll
  for (int i = 0; i < MF_NB; ++i) {
#pragma unroll
    for (int k = i + 1; k < MF_NB; ++k) l[k] -= D[k][i] * l[i];
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < MF_NB; ++i) {
    slot[i * MF_NB + lane] = l[i];
    slot[MF_NB * MF_NB + i * MF_NB + lane] = u[i];
  }
}

// ---------------------------------------------------------------- solves
// 32 contiguous values of a front column (16-byte aligned: ld and the front offsets are
// multiples of 4 elements and k0 of 32)
__device__ __forceinline__ void load_col32(const float* p, float (&v)[MF_NB]) {
#pragma unroll
  for (int q = 0; q < MF_NB / 4; ++q) {
    const float4 t = __ldcg(reinterpret_cast<const float4*>(p) + q);
    v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
  }
}
__device__ __forceinline__ void load_col32(const double* p, double (&v)[MF_NB]) {
#pragma unroll
  for (int q = 0; q < MF_NB / 2; ++q) {
    const double2 t = __ldcg(reinterpret_cast<const double2*>(p) + q);
    v[2 * q] = t.x; v[2 * q + 1] = t.y;
  }
}

struct MFSolveArgs {
  const MFSysDev* sys;
  int nsys;
  const MFFrontDev* fronts;
  int nfront;
  const int32_t* rows;
  const int32_t* relmap;
  const int* done;
  int* sched;
  int* fflag;   // forward done, per front
  int* bflag;   // backward done, per front
};

template <typename T, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
    mf_solve_kernel(MFSolveArgs A, const T* __restrict__ Fall, const T* __restrict__ dinv,
                    const double* __restrict__ rhs, double* __restrict__ x, int accumulate, T* __restrict__ yv,
                    T* __restrict__ dvec, T* __restrict__ upd) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);
  __shared__ T red[NT / 32][MF_NB];
  __shared__ T blk[MF_NB];
  __shared__ T Dinv[MF_NB * MF_NB];
  __shared__ int s_task, s_any;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int epoch = ld_acquire(&A.sched[2]);
  // a pass after every system has converged takes no task at all (the threads check the
  // systems' done flags side by side)
  {
    int pending = A.done ? 0 : 1;
    if (A.done)
      for (int i = tid; i < A.nsys; i += blockDim.x) pending |= !A.done[A.sys[i].sid];
    pending = __syncthreads_or(pending);
    if (tid == 0) s_any = pending;
  }
  __syncthreads();
  for (; s_any;) {
    const int task = next_task(A.sched, &s_task);
    if (task >= 2 * A.nfront) break;
    const bool fwd = task < A.nfront;
    const int f = fwd ? task : 2 * A.nfront - 1 - task;
    const MFFrontDev& Fd = A.fronts[f];
    const MFSysDev& S = A.sys[Fd.sys];
    if (A.done && A.done[S.sid]) continue;   // converged: the whole tree of this system is skipped
    const T* F = Fall + Fd.f_off;
    const int32_t* rw = A.rows + Fd.rows_off;
    const int m = Fd.m, p = Fd.p;
    T* y = yv + S.x_off;
    T* d = dvec + S.x_off;
    if (fwd) {
      if (tid == 0) {
        if (Fd.nchild > 0) wait_flag(&A.fflag[Fd.child0], epoch);
        if (Fd.nchild > 1) wait_flag(&A.fflag[Fd.child1], epoch);
      }
      __syncthreads();
      const double* r = rhs + S.x_off;
      for (int i = tid; i < m; i += blockDim.x) w[i] = i < p ? (T)r[rw[i]] : T(0);
      __syncthreads();
      for (int c = 0; c < Fd.nchild; ++c) {
        const MFFrontDev& C = A.fronts[c == 0 ? Fd.child0 : Fd.child1];
        const int qc = C.m - C.p;
        const int32_t* rm = A.relmap + C.relmap_off;
        const T* u = upd + C.upd_off;
        for (int i = tid; i < qc; i += blockDim.x) w[rm[i]] += ldcg(u + i);
        __syncthreads();
      }
      for (int k0 = 0, kk = 0; k0 < p; k0 += MF_NB, ++kk) {
        const int kb = min(MF_NB, p - k0);
        const T* Li = dinv + Fd.dinv_off + (int64_t)kk * 2 * MF_NB * MF_NB;
#pragma unroll
        for (int u = 0; u < MF_NB * MF_NB / NT; ++u) Dinv[tid + u * NT] = ldcg(Li + tid + u * NT);
        __syncthreads();
        if (warp == 0) {
          T s = T(0);
#pragma unroll
          for (int c = 0; c < MF_NB; ++c)
            if (c < kb) s += Dinv[lane * MF_NB + c] * w[k0 + c];
          __syncwarp();
          if (lane < kb) w[k0 + lane] = s;
        }
        __syncthreads();
        const int k1 = k0 + kb;
        for (int i = k1 + tid; i < m; i += blockDim.x) {
          T fv[MF_NB];
#pragma unroll
          for (int c = 0; c < MF_NB; ++c) fv[c] = c < kb ? ldcg(F + (int64_t)(k0 + c) * Fd.ld + i) : T(0);
          T s = T(0);
#pragma unroll
          for (int c = 0; c < MF_NB; ++c)
            if (c < kb) s += fv[c] * w[k0 + c];
          w[i] -= s;
        }
        __syncthreads();
      }
      for (int i = tid; i < m; i += blockDim.x) {
        if (i < p) y[rw[i]] = w[i];
        else upd[Fd.upd_off + i - p] = w[i];
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(&A.fflag[f], epoch);
      }
    } else {
      if (tid == 0) {
        wait_flag(&A.fflag[f], epoch);
        if (Fd.parent >= 0) wait_flag(&A.bflag[Fd.parent], epoch);
      }
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) w[i] = i < p ? ldcg(y + rw[i]) : ldcg(d + rw[i]);
      __syncthreads();
      const int nblk = (p + MF_NB - 1) / MF_NB;
      for (int kk = nblk - 1; kk >= 0; --kk) {
        const int k0 = kk * MF_NB;
        const int kb = min(MF_NB, p - k0);
        const int k1 = k0 + kb;
        const T* Ui = dinv + Fd.dinv_off + (int64_t)kk * 2 * MF_NB * MF_NB + MF_NB * MF_NB;
#pragma unroll
        for (int u = 0; u < MF_NB * MF_NB / NT; ++u) Dinv[tid + u * NT] = ldcg(Ui + tid + u * NT);
        // U12 (rows k0 .. k1) times w[k1:m]: thread t takes the columns k1 + t, k1 + t + 128, ...
        // (each 32 contiguous values, vector loads, many in flight) and keeps one partial sum
        // per row; the partials are then added over the threads in a fixed order
        {
          T acc[MF_NB];
#pragma unroll
          for (int c = 0; c < MF_NB; ++c) acc[c] = T(0);
          const bool vec = k0 + MF_NB <= Fd.ld;   // the 32 rows stay inside every column
          for (int j = k1 + tid; j < m; j += NT) {
            const T* col = F + (int64_t)j * Fd.ld + k0;
            T v[MF_NB];
            if (vec) {
              load_col32(col, v);
            } else {
#pragma unroll
              for (int c = 0; c < MF_NB; ++c) v[c] = ldcg(col + (c < kb ? c : 0));
            }
            const T wj = w[j];
#pragma unroll
            for (int c = 0; c < MF_NB; ++c) acc[c] += v[c] * wj;
          }
#pragma unroll
          for (int c = 0; c < MF_NB; ++c)
            if (c >= kb) acc[c] = T(0);
          // transpose-reduce over the warp: after the five halving rounds lane l holds the
          // warp's sum for row l (fixed order)
#pragma unroll
          for (int k = 16; k >= 1; k >>= 1) {
            const bool upper = (lane & k) != 0;
#pragma unroll
            for (int i = 0; i < k; ++i) {
              const T send = upper ? acc[i] : acc[i + k];
              const T keep = upper ? acc[i + k] : acc[i];
              acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, k);
            }
          }
          red[warp][lane] = acc[0];
        }
        __syncthreads();
        if (warp == 0) {
          T z = T(0);
          if (lane < kb) {
            z = w[k0 + lane];
#pragma unroll
            for (int q = 0; q < NT / 32; ++q) z -= red[q][lane];
          }
          blk[lane] = z;
          __syncwarp();
          T xv = T(0);
#pragma unroll
          for (int c = 0; c < MF_NB; ++c)
            if (c < kb) xv += Dinv[lane * MF_NB + c] * blk[c];
          if (lane < kb) w[k0 + lane] = xv;
        }
        __syncthreads();
      }
      double* xo = x + S.x_off;
      for (int i = tid; i < p; i += blockDim.x) {
        d[rw[i]] = w[i];
        xo[rw[i]] = accumulate ? xo[rw[i]] + (double)w[i] : (double)w[i];
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(&A.bflag[f], epoch);
      }
    }
  }
  finish_launch(A.sched);
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
size_t mf_factor_smem(bool) {
  return MF_SMEM;   // fixed part + the front when it fits (one CTA per SM)
}

static int mf_grid(const void* fn, size_t smem, int cap, int threads = MF_THREADS) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  const int g = nsm * (per > 0 ? per : 1);
  return cap > 0 && cap < g ? cap : g;
}

template <typename T>
cudaError_t launch_mf_factor(const MFLaunch& L, int task0, int ntask, T* F, T* dinv, int tc, cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  MFArgs A{L.sys, L.fronts, task0, ntask, L.relmap, L.colptr, L.orig_k, L.orig_ij, L.vals, L.status, L.sched,
           L.fflag};
  const bool use_tc = tc && sizeof(T) == 4;
  const size_t smem = mf_factor_smem<T>(use_tc);
  count_launches(1);
  cudaError_t e;
  if constexpr (sizeof(T) == 4) {
    if (use_tc) {
      auto fn = mf_factor_kernel<T, true>;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      // at most two CTAs per SM (shared memory), each allocating half of the tensor memory
      const int grid = std::min(mf_grid((const void*)fn, smem, L.grid_cap), ntask);
      fn<<<grid, MF_THREADS, smem, st>>>(A, F, dinv);
      return cudaGetLastError();
    }
  }
  auto fn = mf_factor_kernel<T, false>;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(mf_grid((const void*)fn, smem, L.grid_cap), ntask);
  fn<<<grid, MF_THREADS, smem, st>>>(A, F, dinv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mf_dinv(T* dinv, const int64_t* blocks, int nblk, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  count_launches(1);
  mf_dinv_kernel<T><<<(nblk + 7) / 8, 256, 0, st>>>(dinv, blocks, nblk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mf_solve(const MFLaunch& L, const T* F, const T* dinv, const double* r, double* x, int accumulate,
                            const int* done, T* yv, T* dv, T* upd, int m_max, cudaStream_t st) {
  if (L.nfront == 0) return cudaSuccess;
  MFSolveArgs A{L.sys, L.nsys, L.fronts, L.nfront, L.rows, L.relmap, done, L.sched + 4, L.sflag, L.sflag + L.nfront};
  const size_t smem = (size_t)(m_max + 4) * sizeof(T);
  count_launches(1);
  // large fronts: 512 threads per CTA keep more of a front's loads in flight; small fronts:
  // 128, more fronts in flight per SM
  const bool wide = m_max >= MF_SOLVE_WIDE_M;
  auto fn = wide ? mf_solve_kernel<T, 512> : mf_solve_kernel<T, MF_STHREADS>;
  const int nt = wide ? 512 : MF_STHREADS;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(mf_grid((const void*)fn, smem, L.grid_cap, nt), 2 * L.nfront);
  fn<<<grid, nt, smem, st>>>(A, F, dinv, r, x, accumulate, yv, dv, upd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mf_big(const MFLaunch& L, const int32_t* list, int nlist, int max_p, int max_m, T* F, T* dinv,
                          int tc, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (nlist > MF_BIG_LIST) return cudaErrorInvalidValue;
  MFBigArgs A{L.sys, L.fronts, list, nlist, L.relmap, L.colptr, L.orig_k, L.orig_ij, L.vals, L.status};
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // CTAs per front for the assembly passes: enough to cover the device several times
  const int per_asm = std::max(1, std::min(256, (8 * nsm + nlist - 1) / nlist));
  for (int phase : {0, 3, 1, 2}) {
    count_launches(1);
    mf_big_assemble_kernel<T><<<dim3(per_asm, nlist), MF_THREADS, 0, st>>>(A, F, phase);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const bool use_tc = tc && sizeof(T) == 4;
  const size_t smem = use_tc ? sizeof(BigUSmem) : (size_t)2 * MF_NB * (MF_TILE + 4) * sizeof(T);
  auto ufn = use_tc ? mf_big_update_kernel<T, true> : mf_big_update_kernel<T, false>;
  const int uthreads = use_tc ? MF_BIG_UTHREADS : MF_THREADS;
  e = cudaFuncSetAttribute(ufn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ugrid = mf_grid((const void*)ufn, smem, L.grid_cap, uthreads);
  for (int k0 = 0; k0 < max_p; k0 += MF_NB) {
    // CTAs per front for the panel: one L21 row or U12 column per thread at most (every CTA
    // of a front repeats the pivot-block factorisation, so no more CTAs than that)
    const int rows = 2 * std::max(0, max_m - k0);
    const int per = std::max(1, std::min(64, (rows + MF_THREADS - 1) / MF_THREADS));
    count_launches(1);
    mf_big_panel_kernel<T><<<dim3(per, nlist), MF_THREADS, 0, st>>>(A, F, dinv, k0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (k0 + MF_NB < max_p) {   // the last pivot block leaves nothing for the next one
      // within a group: its own panels; after its last pivot block: the rest of the trailing
      // region but the Schur block (the group's panels are then complete)
      const int mode = (k0 + MF_NB) % MF_BIG_GROUP == 0 ? 3 : 1;
      count_launches(1);
      ufn<<<ugrid, uthreads, smem, st>>>(A, F, k0, mode);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  count_launches(1);
  ufn<<<ugrid, uthreads, smem, st>>>(A, F, 0, 2);
  return cudaGetLastError();
}

#define TPNS_MF_INST(T)                                                                                      \
  template size_t mf_factor_smem<T>(bool);                                                                  \
  template cudaError_t launch_mf_factor<T>(const MFLaunch&, int, int, T*, T*, int, cudaStream_t);          \
  template cudaError_t launch_mf_dinv<T>(T*, const int64_t*, int, cudaStream_t);                            \
  template cudaError_t launch_mf_big<T>(const MFLaunch&, const int32_t*, int, int, int, T*, T*, int, cudaStream_t); \
  template cudaError_t launch_mf_solve<T>(const MFLaunch&, const T*, const T*, const double*, double*, int, \
                                          const int*, T*, T*, T*, int, cudaStream_t);
TPNS_MF_INST(float)
TPNS_MF_INST(double)

}  // namespace tpns
