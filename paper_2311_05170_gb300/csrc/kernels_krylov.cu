// Restarted GMRES on the local systems, preconditioned by their low-precision factors: the
// fallback of iterative refinement when the classic correction x += (LU)^{-1} r stagnates
// (GMRES-based iterative refinement).  Vectors and the small Hessenberg problem are FP64;
// the preconditioner is the factorisation's own solve.  One CTA per system for every
// reduction (fixed order: deterministic); every kernel skips systems whose skip word is set.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace tpns {
namespace {

constexpr int KT = 256;

// sum over the CTA in a fixed order; every thread gets the result
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = KT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// w = A v (FP64 CSR), four lanes per row
__global__ void __launch_bounds__(KT) spmv_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                  const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                                  const double* __restrict__ vals, const double* __restrict__ v,
                                                  double* __restrict__ w, const int* __restrict__ skip) {
  const int sid = list[blockIdx.y];
  if (skip[sid]) return;
  const SysDev S = sys[sid];
  const int32_t* rp = rowptr + S.rp_off;
  const int32_t* ci = colidx + S.nnz_off;
  const double* va = vals + S.val_off;
  const double* vv = v + S.x_off;
  double* ww = w + S.x_off;
  const int chunk = (S.n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * chunk, r1 = min(S.n, r0 + chunk);
  const int sl = threadIdx.x & 3, slot = threadIdx.x >> 2, per = KT >> 2;
  for (int i0 = r0; i0 < r1; i0 += per) {
    const int i = i0 + slot;
    double acc = 0.0;
    if (i < r1) {
      const int k1 = rp[i + 1];
      for (int k = rp[i] + sl; k < k1; k += 4) acc += va[k] * vv[ci[k]];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (sl == 0 && i < r1) ww[i] = acc;
  }
}

// per system: beta = ||v0||, v0 /= beta, g = beta e_1
__global__ void __launch_bounds__(KT) gm_begin_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                      double* __restrict__ V, int64_t vstride, double* __restrict__ gm,
                                                      int gstride, int kdim, const int* __restrict__ skip) {
  __shared__ double red[KT];
  const int q = blockIdx.x, sid = list[q];
  if (skip[sid]) return;
  const SysDev S = sys[sid];
  double* v0 = V + S.x_off;
  double s = 0;
  for (int i = threadIdx.x; i < S.n; i += KT) s += v0[i] * v0[i];
  const double beta = sqrt(block_sum(s, red));
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  for (int i = threadIdx.x; i < S.n; i += KT) v0[i] *= inv;
  double* G = gm + (int64_t)q * gstride;
  if (threadIdx.x == 0) {
    for (int i = 0; i < gstride; ++i) G[i] = 0.0;
    G[(kdim + 1) * kdim] = beta;   // g[0]
  }
  (void)vstride;
}

// Arnoldi step j: z = V[j+1] (= M^{-1} A V[j]) orthogonalised against V[0..j] (modified
// Gram-Schmidt), normalised; column j of H rotated by the previous Givens rotations, a new
// rotation zeroes H[j+1][j], g rotated with it.
// gm layout per system: H (kdim+1) x kdim row-major, g (kdim+1), cs (kdim), sn (kdim)
__global__ void __launch_bounds__(KT) gm_arnoldi_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                        double* __restrict__ V, int64_t vstride,
                                                        double* __restrict__ gm, int gstride, int kdim, int j,
                                                        const int* __restrict__ skip) {
  __shared__ double red[KT];
  __shared__ double hcol[64];
  const int q = blockIdx.x, sid = list[q];
  if (skip[sid]) return;
  const SysDev S = sys[sid];
  double* z = V + (int64_t)(j + 1) * vstride + S.x_off;
  for (int i = 0; i <= j; ++i) {
    const double* vi = V + (int64_t)i * vstride + S.x_off;
    double s = 0;
    for (int t = threadIdx.x; t < S.n; t += KT) s += z[t] * vi[t];
    const double h = block_sum(s, red);
    for (int t = threadIdx.x; t < S.n; t += KT) z[t] -= h * vi[t];
    if (threadIdx.x == 0) hcol[i] = h;
    __syncthreads();
  }
  double s = 0;
  for (int t = threadIdx.x; t < S.n; t += KT) s += z[t] * z[t];
  const double hn = sqrt(block_sum(s, red));
  const double inv = hn > 0 ? 1.0 / hn : 0.0;
  for (int t = threadIdx.x; t < S.n; t += KT) z[t] *= inv;
  if (threadIdx.x == 0) {
    double* G = gm + (int64_t)q * gstride;
    double* H = G;
    double* g = G + (kdim + 1) * kdim;
    double* cs = g + kdim + 1;
    double* sn = cs + kdim;
    hcol[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = hcol[i], b = hcol[i + 1];
      hcol[i] = cs[i] * a + sn[i] * b;
      hcol[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double a = hcol[j], b = hcol[j + 1];
    const double r = sqrt(a * a + b * b);
    const double c = r > 0 ? a / r : 1.0, sj = r > 0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = sj;
    hcol[j] = r;
    hcol[j + 1] = 0.0;
    const double gj = g[j];
    g[j] = c * gj;
    g[j + 1] = -sj * gj;
    for (int i = 0; i <= j + 1; ++i) H[i * kdim + j] = hcol[i];
  }
}

// x += V[0..k-1] y with H[0..k-1][0..k-1] y = g[0..k-1] (upper triangular after the
// rotations)
__global__ void __launch_bounds__(KT) gm_finish_kernel(const SysDev* __restrict__ sys, const int* __restrict__ list,
                                                       const double* __restrict__ V, int64_t vstride,
                                                       const double* __restrict__ gm, int gstride, int kdim,
                                                       double* __restrict__ x, const int* __restrict__ skip) {
  __shared__ double y[64];
  const int q = blockIdx.x, sid = list[q];
  if (skip[sid]) return;
  const SysDev S = sys[sid];
  if (threadIdx.x == 0) {
    const double* H = gm + (int64_t)q * gstride;
    const double* g = H + (kdim + 1) * kdim;
    for (int i = kdim - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < kdim; ++c) s -= H[i * kdim + c] * y[c];
      const double d = H[i * kdim + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
  }
  __syncthreads();
  double* xx = x + S.x_off;
  for (int t = threadIdx.x; t < S.n; t += KT) {
    double acc = 0.0;
    for (int i = 0; i < kdim; ++i) acc += y[i] * V[(int64_t)i * vstride + S.x_off + t];
    xx[t] += acc;
  }
}

}  // namespace

cudaError_t launch_spmv(const SysDev* sys, const int* list, int nsys, const int32_t* rowptr, const int32_t* colidx,
                        const double* vals, const double* v, double* w, const int* skip, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  spmv_kernel<<<dim3(RES_CHUNKS, nsys), KT, 0, st>>>(sys, list, rowptr, colidx, vals, v, w, skip);
  return cudaGetLastError();
}

cudaError_t launch_gm_begin(const SysDev* sys, const int* list, int nsys, double* V, int64_t vstride, double* gm,
                            int gstride, int kdim, const int* skip, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  gm_begin_kernel<<<nsys, KT, 0, st>>>(sys, list, V, vstride, gm, gstride, kdim, skip);
  return cudaGetLastError();
}

cudaError_t launch_gm_arnoldi(const SysDev* sys, const int* list, int nsys, double* V, int64_t vstride, double* gm,
                              int gstride, int kdim, int j, const int* skip, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  if (kdim > 63) return cudaErrorInvalidValue;
  count_launches(1);
  gm_arnoldi_kernel<<<nsys, KT, 0, st>>>(sys, list, V, vstride, gm, gstride, kdim, j, skip);
  return cudaGetLastError();
}

cudaError_t launch_gm_finish(const SysDev* sys, const int* list, int nsys, const double* V, int64_t vstride,
                             const double* gm, int gstride, int kdim, double* x, const int* skip, cudaStream_t st) {
  if (nsys == 0) return cudaSuccess;
  count_launches(1);
  gm_finish_kernel<<<nsys, KT, 0, st>>>(sys, list, V, vstride, gm, gstride, kdim, x, skip);
  return cudaGetLastError();
}

}  // namespace tpns
