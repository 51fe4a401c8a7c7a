// Launch wrappers of the device kernels (host-callable).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"
#include "mf.hpp"

namespace tpns {

// number of kernel launches issued by this library since it was loaded
int64_t launch_counter();
int64_t thread_launch_counter();   // launches issued by the calling host thread
void count_launches(int n);

constexpr int LU_NB = 32;        // panel width of the band LU and block size of the solves
constexpr int RES_CHUNKS = 64;   // CTAs per system in the residual kernel
constexpr int LU_CLUSTER = 8;    // CTAs per system in the band LU
constexpr int LU_WIDE_CLUSTER_KL = 600;   // bands wider than this get 2 x LU_CLUSTER CTAs where possible

// ---- band linear algebra (kernels_band.cu); `T` = float or double
template <typename T>
cudaError_t launch_band_fill(const SysDev* sys, const int* sys_list, int nsys, const int32_t* rowof,
                             const int32_t* colidx, const double* vals, T* band, int chol,
                             int64_t total_nnz_hint, cudaStream_t st, const int* skip);
template <typename T>
// Unpivoted band LU A = L U into the factor slabs (lslab, uslab), the inverses of the
// diagonal blocks' unit-lower triangles (first half of each block's dinv) and the factored
// diagonal blocks (in the band; launch_band_dinv then forms both inverses from them).
// epoch: device counter, bumped before the factorisation starts
cudaError_t launch_band_lu(const SysDev* sys, const int* sys_list, int nsys, int kl_max, T* band, T* lslab,
                           T* uslab, T* dinv, int* sync, int sync_stride, int* epoch, int* status, cudaStream_t st,
                           const int* skip, int tc = 0, int cl_force = 0);
// tc (FP32 bands): trailing updates on the tensor cores, 1 = TF32 split operands, 2 = plain BF16;
// cl_force: CTAs per cluster (8 or 16, 16 only where all clusters fit; 0 = by band width)
template <typename T>
cudaError_t launch_band_dinv(const SysDev* sys, const int* sys_list, int nsys, int nblk_max, const T* band,
                             T* dinv, cudaStream_t st, const int* skip);
template <typename T>
cudaError_t launch_band_to_slab(const SysDev* sys, const int* sys_list, int nsys, const T* band, T* lslab,
                                T* uslab, cudaStream_t st);
template <typename T>
cudaError_t launch_band_chol(const SysDev* sys, const int* sys_list, int nsys, T* band, int* status,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_chol_to_lu(const SysDev* sys_chol, const SysDev* sys_lu, const int* list, int nsys,
                              const T* cband, T* lband, cudaStream_t st);
// x (+)= U^{-1} L^{-1} r from the factor slabs and the diagonal-block inverses
template <typename T>
cudaError_t launch_band_solve(const SysDev* sys, const int* sys_list, int nsys, int n_max, int kmax,
                              const T* lslab, const T* uslab, const T* dinv, const double* r, double* x,
                              int accumulate, const int* done, int* status, cudaStream_t st, const int* skip,
                              T* vwork = nullptr);
// vwork: scratch in precision T at the systems' x offsets, used when a vector does not fit
// in shared memory beside the pipeline stages (NULL: such a launch fails)
template <typename T>
bool band_solve_fits_smem(int n_max, int kmax);
// dynamic shared memory of the LU kernel for a band of kl_max sub-diagonals
template <typename T>
size_t band_lu_smem_bytes(int kl_max);
// r = b - A x in FP64, convergence bookkeeping (relative residual <= tol, or stagnation);
// first: 0 = a refinement step, 1 = start from x = 0 (r = b), 2 = start from the given x
// partial: nsys * RES_CHUNKS * 2 doubles; ticket: nsys ints, zero before the first call
cudaError_t launch_residual(const SysDev* sys, const int* sys_list, int nsys, const int32_t* rowptr,
                            const int32_t* colidx, const double* vals, const double* b,
                            const double* x, double* r, double* rel, double* rel_prev, int* done,
                            int* iters, double* partial, int* ticket, double tol, int first,
                            cudaStream_t st, const int* skip);

// ---- multifrontal LU of the local Oseen systems (kernels_mf.cu); `T` = float or double
// Factor fronts task0 .. task0 + ntask - 1 of L (all children of a front in the range lie in
// it) in one persistent launch (dataflow over the elimination trees).  tc (float fronts):
// trailing updates on the tensor cores (tcgen05, split TF32).
template <typename T>
cudaError_t launch_mf_factor(const MFLaunch& L, int task0, int ntask, T* F, T* dinv, int tc, cudaStream_t st);
// One refinement pass: x (+)= (LU)^{-1} r for every system of L whose done flag is clear.
// yv, dv: vectors of T at the systems' x offsets; upd: update vectors of the fronts.
template <typename T>
cudaError_t launch_mf_solve(const MFLaunch& L, const T* F, const T* dinv, const double* r, double* x, int accumulate,
                            const int* done, T* yv, T* dv, T* upd, int m_max, cudaStream_t st);
template <typename T>
size_t mf_factor_smem(bool tc);
// Large fronts: factor the listed fronts (one height level of the trees; their children are
// factored) with all CTAs, pivot block by pivot block up to max_p (at most MF_BIG_LIST fronts;
// max_m: their largest order).
template <typename T>
cudaError_t launch_mf_big(const MFLaunch& L, const int32_t* list, int nlist, int max_p, int max_m, T* F, T* dinv,
                          int tc, cudaStream_t st);
// Inverses of the factored pivot blocks (the solves' diagonal blocks): `blocks` lists the
// offsets of the blocks' 2 x 32 x 32 slots in dinv.
template <typename T>
cudaError_t launch_mf_dinv(T* dinv, const int64_t* blocks, int nblk, cudaStream_t st);

// ---- GMRES-based iterative refinement (kernels_krylov.cu); systems with skip[sid] != 0 are
// left alone.  V: kdim + 1 vectors of stride vstride at the systems' x offsets; gm: per
// system (list position) gstride doubles: H ((kdim+1) x kdim), g (kdim+1), cs, sn (kdim each)
cudaError_t launch_spmv(const SysDev* sys, const int* list, int nsys, const int32_t* rowptr, const int32_t* colidx,
                        const double* vals, const double* v, double* w, const int* skip, cudaStream_t st);
cudaError_t launch_gm_begin(const SysDev* sys, const int* list, int nsys, double* V, int64_t vstride, double* gm,
                            int gstride, int kdim, const int* skip, cudaStream_t st);
cudaError_t launch_gm_arnoldi(const SysDev* sys, const int* list, int nsys, double* V, int64_t vstride, double* gm,
                              int gstride, int kdim, int j, const int* skip, cudaStream_t st);
cudaError_t launch_gm_finish(const SysDev* sys, const int* list, int nsys, const double* V, int64_t vstride,
                             const double* gm, int gstride, int kdim, double* x, const int* skip, cudaStream_t st);

// ---- assembly (kernels_assemble.cu)
struct AsmArgs {
  const ProbDev* probs;
  const int32_t* eprob;    // element -> problem
  const double* geo;       // 11 doubles / element
  const int32_t* e6;
  const int32_t* e3;
  const int8_t* egam;
  const int32_t* gnode;    // per local node (n_off)
  const int8_t* nkind;
  const int32_t* gam_src;
  const int32_t* node_dof; // dim per local node
  const int32_t* vloc;     // per local vertex (v_off)
  const int32_t* vert_dof;
  const double* ref;       // reference tables (RefTables or RefTables3, as doubles)
  Phys phys;
  const double* tnow;      // device scalar: t_{n+1}
  int dim;                 // 2: triangles (e6/e3 hold 6/3 per element, geo 11 doubles);
                           // 3: tetrahedra (10/4 per element, geo 22 doubles)
};
cudaError_t launch_oseen_elem(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Ke, double* Re,
                              cudaStream_t st, const int* skip);
cudaError_t launch_darcy_elem(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Re,
                              double* Ke, cudaStream_t st);
// 3D (kernels_assemble3d.cu): element matrices 34 x 34 (Oseen; Re 34 per element) and
// 3 fields x 10 x 10 (Darcy; Re 3 x 10 per element)
cudaError_t launch_oseen_elem3(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Ke, double* Re,
                               cudaStream_t st, const int* skip);
cudaError_t launch_darcy_elem3(const AsmArgs& a, int64_t e_begin, int64_t ne, double* Re, double* Ke,
                               cudaStream_t st);
cudaError_t launch_seg_reduce(const int32_t* tgt, const int32_t* src, int64_t nlanes,
                              const double* in, double* out, cudaStream_t st, const int* skip);
// write e^{n+1} (all local nodes) from the unknowns x
cudaError_t launch_state(const AsmArgs& a, const int32_t* nprob, const int32_t* nvidx,
                         int64_t n_begin, int64_t nn, const double* x, cudaStream_t st,
                         const int* skip);
cudaError_t launch_prolong(int n2c, int n1c, int n2p, const int32_t* pc2i, const double* pc2w,
                           const int32_t* pc1i, const double* pc1w, const int32_t* pp2i,
                           const double* pp2w, const double* uc_new, const double* uc_old,
                           const double* pc_new, const double* pd_new, const double* pd_old,
                           int64_t nnpH, double* FW1, double* FW0, double* FP1, double* FPD1,
                           double* FPD0, int64_t nnp, cudaStream_t st, int dim = 2);
struct GlueArgs {
  const ProbDev* fluid;
  const ProbDev* porous;
  const int32_t *gc_ptr, *gc_prob, *gc_node; const double* gc_w;
  const int32_t *gp_ptr, *gp_prob, *gp_node; const double* gp_w;
  const int32_t *gv_ptr, *gv_prob, *gv_vert; const double* gv_w;
  const double *FW1, *FP1, *FPD1;
  double *out_u, *out_p, *out_pd;
  int nnc, nvc, nnp;
  int dim;          // velocity components per node
  int add_coarse;   // 1: add the coarse interpolant (one rank of a split simulation, or the whole)
};
cudaError_t launch_glue(const GlueArgs& g, cudaStream_t st);
// coarse Newton: u += delta (all coarse nodes), p += delta_p; convergence flag
cudaError_t launch_newton_update(const ProbDev* prob, const int32_t* gnode, const int32_t* vloc,
                                 int nn, int nvl, double* u, double* p, int* done, int* iters,
                                 cudaStream_t st);
// x <- 2 x - xprev once *step >= 2 (else x unchanged), xprev <- the old x: initial local iterates
cudaError_t launch_predict(double* x, double* xprev, int64_t n, const int64_t* step, cudaStream_t st);
cudaError_t launch_set_time(double* tnow, int64_t* step, double dt, int advance, cudaStream_t st);

}  // namespace tpns
