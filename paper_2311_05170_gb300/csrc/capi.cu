// Context and C ABI of the GB300 library (declared in tpns.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <atomic>
#include <chrono>
#include <mutex>
#include <array>
#include <vector>

#include "kernels.hpp"
#include "setup.hpp"
#include "tpns.h"

using namespace tpns;

// Phases timed with CUDA events on the context's stream when timing is enabled.
enum Phase {
  PH_COARSE = 0, PH_PROLONG, PH_ASM_OSEEN, PH_SCATTER, PH_ASM_DARCY, PH_BAND_FILL, PH_BAND_LU,
  PH_SOLVE, PH_RESIDUAL, PH_STATE_GLUE, PH_COPIES, PH_COUNT
};

struct tpns_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  tpns_precision prec = TPNS_FP64;
  double dt = 0;
  Phys phys{};
  Layout L;
  RefTables ref{};
  RefTables3 ref3{};
  // element shape: dimension, Oseen / Darcy slots per element, P2 nodes and vertices per
  // element, geometry doubles per element
  int dim = 2, SO = 15, SD = 6, NPE = 6, VPE = 3, GEO = 11;
  std::string err;
  std::vector<void*> allocs;
  size_t bytes = 0;
  size_t budget = 0;   // cap on `bytes` (0: none); every allocation is checked against it
  // problems: fluid locals [0,nf), CF = nf, porous locals [nf+1, nf+1+np), CP = nf+1+np
  int nf = 0, np = 0, nprob = 0;
  std::vector<const Problem*> probs;
  std::vector<ProbDev> hprob;
  std::vector<int64_t> e_off, n_off, v_off, x_off;
  std::vector<int> sys_first;             // first system of a problem
  int64_t ne_tot = 0, nn_tot = 0, nv_tot = 0;
  int64_t ne_osl = 0, ne_cf = 0, eD0 = 0, ne_dl = 0, ne_cp = 0;   // element ranges
  int64_t nn_fl = 0, nn_cf = 0, nn_pl = 0, nn_cp = 0;              // node ranges (begins below)
  int64_t nb_fl = 0, nb_cf = 0, nb_pl = 0, nb_cp = 0;
  // systems
  std::vector<SysDev> hsys;
  std::vector<int> hchol;
  int nsys = 0;
  std::vector<int> list_osl, list_cf, list_dl, list_cp, list_local;
  int kl_max_osl = 0, n_max_local = 0, kmax_local = 0, kmax_cf = 0, kmax_cp = 0, kl_max_cf = 0, n_max_cf = 0, n_max_cp = 0;
  int64_t band_local_len = 0, band_coarse_len = 0, nnz_tot = 0, vals_tot = 0, xvec_tot = 0;
  double lu_flops_step = 0;
  std::vector<SysDev> hsys_chol;          // Cholesky layout of the Darcy systems (setup only)
  int64_t band_chol_local_len = 0, band_chol_coarse_len = 0, dinv_local_len = 0, dinv_coarse_len = 0;
  int64_t lslab_local_len = 0, uslab_local_len = 0, lslab_coarse_len = 0, uslab_coarse_len = 0;
  int nblk_max_osl = 1, nblk_max_dl = 1, nblk_max_cf = 1, nblk_max_cp = 1;
  int flags_stride = 1;
  bool host_only = false;
  // CUDA graphs of one step: coarse solve + hot path, and hot path alone
  bool use_graph = true;
  bool own_stream = false;
  cudaGraphExec_t g_full = nullptr, g_local = nullptr;
  int64_t kernels_full = 0, kernels_local = 0;   // kernels in each captured graph
  cudaEvent_t ev_s0 = nullptr, ev_s1 = nullptr;   // bracket the context's step in tpns_batch_step
  int lu_cl = 0;                                   // CTAs per cluster of the Oseen LU, picked at create
  // multifrontal factorisation of the local Oseen systems
  bool mf = false;
  int mf_leaf = 96, mf_tc = 1, mf_m_max = 1, mf_oseen_fronts = 0;
  // large fronts (factored by all CTAs): order threshold, fronts of the dataflow launch per
  // group (Oseen, Darcy), and per group the height levels (offset into d_mf_big, count, max p)
  int mf_big_m = 256;
  int mf_small[2] = {0, 0};
  std::vector<std::array<int, 4>> mf_big_levels[2];   // (offset in the list, fronts, max p, max m)
  int32_t* d_mf_big = nullptr;
  int mf_oseen_blocks = 0, mf_blocks = 0;   // pivot blocks of the Oseen fronts / of all fronts
  int64_t* d_mf_dblk = nullptr;
  int rank = 0, nranks = 1;   // split of one simulation over contexts (see tpns_options)
  bool alg1 = false;          // Algorithm 1: the coarse mesh is the fine mesh, no local phase
  bool gmres = false;         // GMRES-based refinement when classic refinement stagnates
  int ir_classic_max = 0;     // classic refinement passes per step (0: default)
  double *gm_V = nullptr, *gm_W = nullptr, *gm_H = nullptr;
  int* gm_skip = nullptr;
  double mf_flops = 0, mf_factor_entries = 0, mf_dinv_entries = 0;
  MFLaunch mfl{};
  std::vector<MFSysDev> h_mfsys;
  int64_t mf_F_len = 0, mf_dinv_len = 0, mf_upd_len = 0;
  void *d_mf_F = nullptr, *d_mf_dinv = nullptr, *d_mf_y = nullptr, *d_mf_d = nullptr, *d_mf_upd = nullptr;
  // band solves: every local system (band LU) or the Darcy systems only (multifrontal)
  std::vector<int> list_band;
  int* d_list_band = nullptr;
  int n_max_band = 0, kmax_band = 0;
  // device
  ProbDev* d_probs = nullptr;
  int32_t *d_eprob = nullptr, *d_e6 = nullptr, *d_e3 = nullptr;
  int8_t* d_egam = nullptr;
  double* d_geo = nullptr;
  int32_t *d_gnode = nullptr, *d_gam_src = nullptr, *d_node_dof = nullptr, *d_nprob = nullptr, *d_nvidx = nullptr;
  int8_t* d_nkind = nullptr;
  int32_t *d_vloc = nullptr, *d_vert_dof = nullptr;
  double* d_ref = nullptr;
  SysDev* d_sys = nullptr;
  int* d_chol = nullptr;
  int32_t *d_rowptr = nullptr, *d_colidx = nullptr, *d_rowof = nullptr;
  double* d_vals = nullptr;
  double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr, *d_rel = nullptr, *d_relprev = nullptr;
  int *d_done = nullptr, *d_iters = nullptr, *d_status = nullptr, *d_ticket = nullptr;
  double* d_partial = nullptr;
  void* d_band_local = nullptr;
  double* d_band_coarse = nullptr;
  void* d_dinv_local = nullptr;
  void* d_vwork = nullptr;   // solve vectors that do not fit in shared memory (precision T), or NULL
  double* d_dinv_coarse = nullptr;
  void *d_lslab_local = nullptr, *d_uslab_local = nullptr;
  double *d_lslab_coarse = nullptr, *d_uslab_coarse = nullptr;
  // FP32 factors of the coarse conduit Jacobian (FP32_IR contexts): band, slabs, inverses at
  // the same element offsets as the FP64 coarse buffers
  float *d_band_coarse_f = nullptr, *d_lslab_coarse_f = nullptr, *d_uslab_coarse_f = nullptr,
        *d_dinv_coarse_f = nullptr;
  int* d_flags = nullptr;
  int* d_epoch = nullptr;
  SysDev* d_sys_chol = nullptr;
  int *d_list_osl = nullptr, *d_list_cf = nullptr, *d_list_dl = nullptr, *d_list_cp = nullptr,
      *d_list_local = nullptr;
  double *d_Ke = nullptr, *d_Re = nullptr, *d_ReD = nullptr;
  int32_t *d_mo_t = nullptr, *d_mo_s = nullptr, *d_ro_t = nullptr, *d_ro_s = nullptr;
  int32_t *d_rd_t = nullptr, *d_rd_s = nullptr;
  int32_t *d_mcf_t = nullptr, *d_mcf_s = nullptr, *d_rcf_t = nullptr, *d_rcf_s = nullptr;
  int32_t *d_rcp_t = nullptr, *d_rcp_s = nullptr;
  int64_t n_mo = 0, n_ro = 0, n_rd = 0, n_mcf = 0, n_rcf = 0, n_rcp = 0;
  double *d_uc_old = nullptr, *d_uc_new = nullptr, *d_pc_new = nullptr, *d_pd_old = nullptr,
         *d_pd_new = nullptr, *d_zero = nullptr, *d_delta = nullptr;
  double *d_FW1 = nullptr, *d_FW0 = nullptr, *d_FP1 = nullptr, *d_FPD1 = nullptr, *d_FPD0 = nullptr;
  double *d_out_u = nullptr, *d_out_p = nullptr, *d_out_pd = nullptr;
  int32_t *d_pc2i = nullptr, *d_pc1i = nullptr, *d_pp2i = nullptr;
  double *d_pc2w = nullptr, *d_pc1w = nullptr, *d_pp2w = nullptr;
  int32_t *d_gc_ptr = nullptr, *d_gc_prob = nullptr, *d_gc_node = nullptr;
  int32_t *d_gp_ptr = nullptr, *d_gp_prob = nullptr, *d_gp_node = nullptr;
  int32_t *d_gv_ptr = nullptr, *d_gv_prob = nullptr, *d_gv_vert = nullptr;
  double *d_gc_w = nullptr, *d_gp_w = nullptr, *d_gv_w = nullptr;
  double* d_tnow = nullptr;
  int64_t* d_step = nullptr;
  double* d_xprev = nullptr;
  int *d_newton_done = nullptr, *d_newton_iters = nullptr;
  // coarse trajectory for tpns_local_step
  std::vector<double*> traj;          // per stored step: uc, pc, pd (concatenated)
  int64_t traj_len = 0;
  int traj_base = 0;                  // step index of traj[0]
  int64_t step = 0;
  tpns_stats stats{};
  // phase timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  cudaEvent_t ev_open[PH_COUNT] = {};
  double ph_ms[PH_COUNT] = {};
  int64_t ph_n[PH_COUNT] = {};
  AsmArgs asmargs{};
  GlueArgs glue{};
};

// message of the last failure raised without a context (per host thread, so concurrent
// callers do not overwrite each other's message)
static thread_local std::string g_err;


static void ph_begin(tpns_ctx* ctx, int id);
static void ph_end(tpns_ctx* ctx, int id);

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
      return TPNS_EDEVICE;                                                         \
    }                                                                              \
  } while (0)

template <typename T>
static tpns_status dalloc(tpns_ctx* ctx, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (ctx->budget > 0 && ctx->bytes + n * sizeof(T) > ctx->budget) {
    ctx->err = "device footprint exceeds the budget of " + std::to_string(ctx->budget) + " B";
    return TPNS_EBUDGET;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return TPNS_ENOMEM;
  }
  ctx->allocs.push_back(q);
  ctx->bytes += n * sizeof(T);
  *p = reinterpret_cast<T*>(q);
  return TPNS_OK;
}

template <typename T>
static tpns_status upload(tpns_ctx* ctx, T** p, const std::vector<T>& v) {
  tpns_status s = dalloc(ctx, p, v.size());
  if (s != TPNS_OK) return s;
  ctx->stats.h2d_bytes += (int64_t)(v.size() * sizeof(T));
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TPNS_OK;
}

#define TRY(x)                      \
  do {                              \
    tpns_status s_ = (x);           \
    if (s_ != TPNS_OK) return s_;   \
  } while (0)

// ------------------------------------------------------------------------------ host data
static void mms_u_host(const Phys& P, double x, double y, double t, double* u) {
  if (P.mms == 1) {
    const double pi = 3.141592653589793;
    double E = std::exp(-t);
    u[0] = std::sin(pi * x) * std::cos(pi * y) * E;
    u[1] = -std::cos(pi * x) * std::sin(pi * y) * E;
  } else if (P.mms == 3) {
    u[0] = x * x;
    u[1] = -2.0 * x * y;
  } else {
    u[0] = u[1] = 0.0;
  }
}
static double mms_p_host(const Phys& P, double x, double y, double t) {
  const double pi = 3.141592653589793;
  if (P.mms == 1) return std::cos(pi * x) * std::cos(pi * y) * std::exp(-t);
  if (P.mms == 3) return x + y;
  return 0.0;
}
static double mms_pd_host(const Phys& P, int f, double x, double y, double t) {
  const double pi = 3.141592653589793;
  const double a = 3.0 - f;
  if (P.mms == 1) return a * std::cos(pi * x) * std::cos(pi * y) * std::exp(-t);
  if (P.mms == 3) return a * (x * x + y * y);
  return 0.0;
}

// 3D manufactured fields (mms 2: trigonometric, 4: polynomial patch; see device.cuh)
static void mms3_u_host(const Phys& P, const double* X, double t, double* u) {
  const double pi = 3.141592653589793;
  const double x = X[0], y = X[1], z = X[2];
  if (P.mms == 2) {
    const double E = std::exp(-t);
    u[0] = std::sin(pi * x) * std::cos(pi * y) * std::cos(pi * z) * E;
    u[1] = std::cos(pi * x) * std::sin(pi * y) * std::cos(pi * z) * E;
    u[2] = -2.0 * std::cos(pi * x) * std::cos(pi * y) * std::sin(pi * z) * E;
  } else if (P.mms == 4) {
    u[0] = x * x; u[1] = y * y; u[2] = -2.0 * (x + y) * z;
  } else {
    u[0] = u[1] = u[2] = 0.0;
  }
}
static double mms3_p_host(const Phys& P, const double* X, double t) {
  const double pi = 3.141592653589793;
  if (P.mms == 2) return std::cos(pi * X[0]) * std::cos(pi * X[1]) * std::cos(pi * X[2]) * std::exp(-t);
  if (P.mms == 4) return X[0] + X[1] + X[2];
  return 0.0;
}
static double mms3_pd_host(const Phys& P, int f, const double* X, double t) {
  const double a = 3.0 - f;
  const double pi = 3.141592653589793;
  if (P.mms == 2) return a * std::cos(pi * X[0]) * std::cos(pi * X[1]) * std::cos(pi * X[2]) * std::exp(-t);
  if (P.mms == 4) return a * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  return 0.0;
}
// velocity / pressure / Darcy pressure of the manufactured solution at node i of a mesh
static void mms_u_node(const tpns_ctx* ctx, const Mesh& m, int i, double t, double* u) {
  if (ctx->dim == 3) mms3_u_host(ctx->phys, &m.node[3 * (size_t)i], t, u);
  else mms_u_host(ctx->phys, m.node[2 * (size_t)i], m.node[2 * (size_t)i + 1], t, u);
}
static double mms_p_node(const tpns_ctx* ctx, const Mesh& m, int i, double t) {
  if (ctx->dim == 3) return mms3_p_host(ctx->phys, &m.node[3 * (size_t)i], t);
  return mms_p_host(ctx->phys, m.node[2 * (size_t)i], m.node[2 * (size_t)i + 1], t);
}
static double mms_pd_node(const tpns_ctx* ctx, int f, const Mesh& m, int i, double t) {
  if (ctx->dim == 3) return mms3_pd_host(ctx->phys, f, &m.node[3 * (size_t)i], t);
  return mms_pd_host(ctx->phys, f, m.node[2 * (size_t)i], m.node[2 * (size_t)i + 1], t);
}

static std::vector<int32_t> inverse_map(const std::vector<int32_t>& g, int n) {
  std::vector<int32_t> inv(n, -1);
  for (size_t l = 0; l < g.size(); ++l) inv[g[l]] = (int32_t)l;
  return inv;
}

// ------------------------------------------------------------------------------ create
static tpns_status build_ctx(tpns_ctx* ctx, const tpns_mesh_desc& md, const tpns_partition_desc& pd,
                             size_t budget) {
  Layout& L = ctx->L;
  std::string msg = build_layout(md, pd, L, ctx->mf ? ctx->mf_leaf : 0, ctx->rank, ctx->nranks);
  if (!msg.empty()) {
    ctx->err = msg;
    return TPNS_EINVAL;
  }
  ctx->dim = L.dim;
  if (ctx->dim == 3) {
    build_ref_tables3(ctx->ref3);
    ctx->SO = 34; ctx->SD = 10; ctx->NPE = 10; ctx->VPE = 4; ctx->GEO = 22;
  } else {
    build_ref_tables(ctx->ref);
  }
  ctx->nf = (int)L.fluid.size();
  ctx->np = (int)L.porous.size();
  ctx->probs.clear();
  for (auto& P : L.fluid) ctx->probs.push_back(&P);
  ctx->probs.push_back(&L.cfl);
  for (auto& P : L.porous) ctx->probs.push_back(&P);
  ctx->probs.push_back(&L.cpo);
  ctx->nprob = (int)ctx->probs.size();
  const int CF = ctx->nf, CP = ctx->nf + 1 + ctx->np;
  // offsets
  int64_t e = 0, n = 0, v = 0;
  ctx->e_off.resize(ctx->nprob);
  ctx->n_off.resize(ctx->nprob);
  ctx->v_off.resize(ctx->nprob);
  for (int p = 0; p < ctx->nprob; ++p) {
    ctx->e_off[p] = e; ctx->n_off[p] = n; ctx->v_off[p] = v;
    e += ctx->probs[p]->ne; n += ctx->probs[p]->nn; v += ctx->probs[p]->nvl;
  }
  ctx->ne_tot = e; ctx->nn_tot = n; ctx->nv_tot = v;
  ctx->ne_osl = ctx->e_off[CF];
  ctx->ne_cf = ctx->probs[CF]->ne;
  ctx->eD0 = ctx->e_off[CF + 1 < ctx->nprob ? CF + 1 : CF];
  ctx->ne_dl = ctx->e_off[CP] - ctx->eD0;
  ctx->ne_cp = ctx->probs[CP]->ne;
  ctx->nb_fl = 0; ctx->nn_fl = ctx->n_off[CF];
  ctx->nb_cf = ctx->n_off[CF]; ctx->nn_cf = ctx->probs[CF]->nn;
  ctx->nb_pl = ctx->n_off[CF] + ctx->nn_cf; ctx->nn_pl = ctx->n_off[CP] - ctx->nb_pl;
  ctx->nb_cp = ctx->n_off[CP]; ctx->nn_cp = ctx->probs[CP]->nn;
  // systems
  ctx->hsys.clear(); ctx->hchol.clear(); ctx->hsys_chol.clear(); ctx->sys_first.assign(ctx->nprob, 0);
  ctx->band_chol_local_len = ctx->band_chol_coarse_len = ctx->dinv_local_len = ctx->dinv_coarse_len = 0;
  ctx->lslab_local_len = ctx->uslab_local_len = ctx->lslab_coarse_len = ctx->uslab_coarse_len = 0;
  ctx->x_off.assign(ctx->nprob, 0);
  int64_t rp = 0, nz = 0, vals = 0, xo = 0, bl = 0, bc = 0;
  std::vector<int32_t> h_rowptr, h_colidx, h_rowof;
  ctx->lu_flops_step = 0;
  for (int p = 0; p < ctx->nprob; ++p) {
    const Problem& P = *ctx->probs[p];
    const bool coarse = P.coarse;
    ctx->sys_first[p] = (int)ctx->hsys.size();
    ctx->x_off[p] = xo;
    const int nfld = P.kind == PK_OSEEN ? 1 : 3;
    h_rowptr.insert(h_rowptr.end(), P.rowptr.begin(), P.rowptr.end());
    h_colidx.insert(h_colidx.end(), P.colidx.begin(), P.colidx.end());
    h_rowof.insert(h_rowof.end(), P.rowof.begin(), P.rowof.end());
    for (int f = 0; f < nfld; ++f) {
      SysDev S{};
      S.n = P.n; S.kl = P.kl; S.ku = P.kind == PK_OSEEN ? P.ku : P.kl;
      S.ldab = S.kl + S.ku + 1;
      S.rp_off = rp; S.nnz_off = nz; S.nnz = (int64_t)P.colidx.size();
      S.val_off = vals; vals += S.nnz;
      S.x_off = xo; xo += P.n;
      const int64_t blen = (int64_t)S.n * S.ldab;
      const int nblk = (S.n + LU_NB - 1) / LU_NB;
      const int64_t dlen = (int64_t)nblk * 2 * LU_NB * LU_NB;
      ctx->flags_stride = std::max(ctx->flags_stride, nblk);
      SysDev C = S;
      C.ku = 0; C.ldab = S.kl + 1;
      auto round32 = [](int64_t v) { return (v + 31) & ~(int64_t)31; };
      const int64_t llen = (int64_t)nblk * LU_NB * S.kl, ulen = (int64_t)nblk * LU_NB * S.ku;
      if (coarse) {
        S.band_off = bc; bc += blen;
        S.dinv_off = ctx->dinv_coarse_len; ctx->dinv_coarse_len += dlen;
        C.band_off = ctx->band_chol_coarse_len; ctx->band_chol_coarse_len += (int64_t)S.n * C.ldab;
        S.lslab_off = ctx->lslab_coarse_len; ctx->lslab_coarse_len += round32(llen);
        S.uslab_off = ctx->uslab_coarse_len; ctx->uslab_coarse_len += round32(ulen);
      } else if (ctx->mf) {
        // factored by the multifrontal LU: no band storage
        S.band_off = 0; S.dinv_off = 0; S.lslab_off = 0; S.uslab_off = 0; C.band_off = 0;
      } else {
        S.band_off = bl; bl += blen;
        S.dinv_off = ctx->dinv_local_len; ctx->dinv_local_len += dlen;
        C.band_off = ctx->band_chol_local_len; ctx->band_chol_local_len += (int64_t)S.n * C.ldab;
        S.lslab_off = ctx->lslab_local_len; ctx->lslab_local_len += round32(llen);
        S.uslab_off = ctx->uslab_local_len; ctx->uslab_local_len += round32(ulen);
      }
      ctx->hsys.push_back(S);
      ctx->hsys_chol.push_back(C);
      ctx->hchol.push_back(P.kind == PK_DARCY ? 1 : 0);
    }
    rp += P.n + 1; nz += (int64_t)P.colidx.size();
    if (P.kind == PK_OSEEN && !coarse) ctx->lu_flops_step += ctx->mf ? P.mf.flops : P.lu_flops;
  }
  ctx->nsys = (int)ctx->hsys.size();
  ctx->nnz_tot = nz; ctx->vals_tot = vals; ctx->xvec_tot = xo;
  ctx->band_local_len = bl; ctx->band_coarse_len = bc;
  ctx->list_osl.clear(); ctx->list_dl.clear(); ctx->list_local.clear();
  for (int p = 0; p < ctx->nf; ++p) ctx->list_osl.push_back(ctx->sys_first[p]);
  ctx->list_cf = {ctx->sys_first[CF]};
  for (int p = CF + 1; p < CP; ++p)
    for (int f = 0; f < 3; ++f) ctx->list_dl.push_back(ctx->sys_first[p] + f);
  ctx->list_cp = {ctx->sys_first[CP], ctx->sys_first[CP] + 1, ctx->sys_first[CP] + 2};
  ctx->list_local = ctx->list_osl;
  ctx->list_local.insert(ctx->list_local.end(), ctx->list_dl.begin(), ctx->list_dl.end());
  if (ctx->mf) ctx->list_band.clear();
  else ctx->list_band = ctx->list_local;
  for (int s : ctx->list_band) {
    ctx->n_max_band = std::max(ctx->n_max_band, ctx->hsys[s].n);
    ctx->kmax_band = std::max(ctx->kmax_band, std::max(ctx->hsys[s].kl, ctx->hsys[s].ku));
  }
  for (int s : ctx->list_osl) ctx->kl_max_osl = std::max(ctx->kl_max_osl, ctx->hsys[s].kl);
  for (int s : ctx->list_local) {
    ctx->n_max_local = std::max(ctx->n_max_local, ctx->hsys[s].n);
    ctx->kmax_local = std::max(ctx->kmax_local, std::max(ctx->hsys[s].kl, ctx->hsys[s].ku));
  }
  ctx->kmax_cf = std::max(ctx->hsys[ctx->list_cf[0]].kl, ctx->hsys[ctx->list_cf[0]].ku);
  auto nblk_of = [&](int sidx) { return (ctx->hsys[sidx].n + LU_NB - 1) / LU_NB; };
  for (int sidx : ctx->list_osl) ctx->nblk_max_osl = std::max(ctx->nblk_max_osl, nblk_of(sidx));
  for (int sidx : ctx->list_dl) ctx->nblk_max_dl = std::max(ctx->nblk_max_dl, nblk_of(sidx));
  ctx->nblk_max_cf = nblk_of(ctx->list_cf[0]);
  for (int sidx : ctx->list_cp) ctx->nblk_max_cp = std::max(ctx->nblk_max_cp, nblk_of(sidx));
  for (int s : ctx->list_cp) ctx->kmax_cp = std::max(ctx->kmax_cp, ctx->hsys[s].kl);
  ctx->kl_max_cf = ctx->hsys[ctx->list_cf[0]].kl;
  ctx->n_max_cf = ctx->hsys[ctx->list_cf[0]].n;
  for (int s : ctx->list_cp) ctx->n_max_cp = std::max(ctx->n_max_cp, ctx->hsys[s].n);
  // multifrontal layout of the local systems: the fronts of all systems in one task order
  // per group, in which a front's children always precede it
  std::vector<MFFrontDev> h_fronts;
  std::vector<int64_t> h_dblk;   // pivot-block slots: the Oseen fronts' first, then the Darcy fronts'
  std::vector<int32_t> h_mrows, h_relmap, h_origk, h_origi, h_big;
  std::vector<int64_t> h_colptr;
  if (ctx->mf) {
    ctx->h_mfsys.clear();
    ctx->mf_flops = ctx->mf_factor_entries = ctx->mf_dinv_entries = 0;
    // multifrontal systems: the Oseen systems (factored every step), then the three fields
    // of every porous subdomain (factored once); each group's fronts in level order
    struct MSys { int prob, sid; };
    std::vector<MSys> msys;
    for (int q = 0; q < ctx->nf; ++q) msys.push_back({q, ctx->sys_first[q]});
    for (int q = ctx->nf + 1; q < ctx->nf + 1 + ctx->np; ++q)
      for (int f = 0; f < 3; ++f) msys.push_back({q, ctx->sys_first[q] + f});
    // Task order: a front's priority is the estimated time from its start to the end of its
    // tree's root (its own cost plus its parent's priority), so children always rank before
    // their parents (the order stays topological) and the fronts on the longest remaining
    // chains are taken first.  Estimated cost of a front in microseconds: fixed work plus
    // per-pivot-block work plus the assembly and update traffic.
    // Large fronts (order >= mf_big_m) and all their ancestors go to the large-front path;
    // the others (which then have no large descendant) to the dataflow launch.
    struct Key { int group, big, lvl; double prio; int q, t; };
    std::vector<Key> keys;
    std::vector<std::vector<int>> newid(msys.size());
    for (int q = 0; q < (int)msys.size(); ++q) {
      const MFSymbolic& M = ctx->probs[msys[q].prob]->mf;
      const bool oseen = msys[q].prob < ctx->nf;
      newid[q].assign(M.fronts.size(), -1);
      const int nf = (int)M.fronts.size();
      std::vector<double> prio(nf, 0.0);
      for (int t = nf - 1; t >= 0; --t) {   // postorder: parents after children
        const MFFront& F = M.fronts[t];
        const double cost = 10.0 + 15.0 * ((F.p + MF_NB - 1) / MF_NB) + 1e-3 * (double)F.m * F.m;
        prio[t] = cost + (F.parent >= 0 ? prio[F.parent] : 0.0);
      }
      std::vector<int> height(nf, 0);
      std::vector<char> big(nf, 0);
      for (int t = 0; t < nf; ++t) {
        const MFFront& F = M.fronts[t];
        for (int c = 0; c < F.nchild; ++c) height[t] = std::max(height[t], height[F.child[c]] + 1);
        if (ctx->mf_big_m > 0 && F.m >= ctx->mf_big_m)
          for (int u = t; u >= 0 && !big[u]; u = M.fronts[u].parent) big[u] = 1;
      }
      for (int t = 0; t < nf; ++t) keys.push_back({oseen ? 0 : 1, big[t], big[t] ? height[t] : 0, prio[t], q, t});
      const SysDev& Sd = ctx->hsys[msys[q].sid];
      MFSysDev D{};
      D.sid = msys[q].sid; D.n = ctx->probs[msys[q].prob]->n; D.x_off = Sd.x_off; D.val_off = Sd.val_off;
      ctx->h_mfsys.push_back(D);
      if (oseen) {
        ctx->mf_flops += M.flops;
        ctx->mf_factor_entries += M.factor_entries;
      }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
      if (a.group != b.group) return a.group < b.group;
      if (a.big != b.big) return a.big < b.big;
      if (a.lvl != b.lvl) return a.lvl < b.lvl;
      return a.prio > b.prio;
    });
    ctx->mf_oseen_fronts = 0;
    ctx->mf_small[0] = ctx->mf_small[1] = 0;
    ctx->mf_big_levels[0].clear();
    ctx->mf_big_levels[1].clear();
    h_big.clear();
    for (size_t i = 0; i < keys.size(); ++i) {
      newid[keys[i].q][keys[i].t] = (int)i;
      const int g = keys[i].group;
      if (g == 0) ctx->mf_oseen_fronts = (int)i + 1;
      if (!keys[i].big) {
        ctx->mf_small[g] += 1;
        continue;
      }
      auto& lv = ctx->mf_big_levels[g];
      const MFFront& BF = ctx->probs[msys[keys[i].q].prob]->mf.fronts[keys[i].t];
      if (lv.empty() || keys[i - 1].lvl != keys[i].lvl || !keys[i - 1].big || keys[i - 1].group != g ||
          lv.back()[1] >= MF_BIG_LIST)
        lv.push_back({(int)h_big.size(), 0, 0, 0});
      lv.back()[1] += 1;
      lv.back()[2] = std::max(lv.back()[2], BF.p);
      lv.back()[3] = std::max(lv.back()[3], BF.m);
      h_big.push_back((int32_t)i);
    }
    for (const Key& k : keys) {
      const MFFront& F = ctx->probs[msys[k.q].prob]->mf.fronts[k.t];
      if (F.m >= 32768) {
        ctx->err = "a multifrontal front of order " + std::to_string(F.m) + " exceeds 32767";
        return TPNS_EINVAL;
      }
      MFFrontDev FD{};
      FD.m = F.m; FD.p = F.p; FD.ld = (F.m + 3) & ~3; FD.sys = k.q;
      FD.f_off = ctx->mf_F_len; ctx->mf_F_len += (int64_t)FD.ld * F.m;
      const int nb = (F.p + MF_NB - 1) / MF_NB;
      FD.dinv_off = ctx->mf_dinv_len; ctx->mf_dinv_len += (int64_t)nb * 2 * MF_NB * MF_NB;
      FD.upd_off = ctx->mf_upd_len; ctx->mf_upd_len += F.m - F.p;
      FD.nchild = F.nchild;
      FD.child0 = F.nchild > 0 ? newid[k.q][F.child[0]] : -1;
      FD.child1 = F.nchild > 1 ? newid[k.q][F.child[1]] : -1;
      FD.parent = F.parent >= 0 ? newid[k.q][F.parent] : -1;
      FD.rows_off = (int32_t)h_mrows.size();
      h_mrows.insert(h_mrows.end(), F.rows.begin(), F.rows.end());
      FD.relmap_off = (int32_t)h_relmap.size();
      h_relmap.insert(h_relmap.end(), F.relmap.begin(), F.relmap.end());
      FD.colptr_off = (int32_t)h_colptr.size();
      const int64_t ob = (int64_t)h_origk.size();
      for (int j = 0; j <= F.m; ++j) h_colptr.push_back(ob + F.col_ptr[j]);
      h_origk.insert(h_origk.end(), F.orig_k.begin(), F.orig_k.end());
      for (int j = 0; j < F.m; ++j)
        for (int q = F.col_ptr[j]; q < F.col_ptr[j + 1]; ++q) h_origi.push_back(F.orig_i[q] | (j << 16));
      ctx->mf_m_max = std::max(ctx->mf_m_max, F.m);
      if (k.group == 0) ctx->mf_dinv_entries += (double)nb * 2 * MF_NB * MF_NB;
      for (int b = 0; b < nb; ++b) h_dblk.push_back(FD.dinv_off + (int64_t)b * 2 * MF_NB * MF_NB);
      if (k.group == 0) ctx->mf_oseen_blocks = (int)h_dblk.size();
      h_fronts.push_back(FD);
    }
  }
  // footprint check before any allocation
  const size_t Tsz = ctx->prec == TPNS_FP64 ? 8 : 4;
  size_t est = (size_t)ctx->band_local_len * Tsz + (size_t)ctx->band_coarse_len * 8 +
               (size_t)(ctx->ne_osl + ctx->ne_cf) * (ctx->SO * ctx->SO + ctx->SO) * 8 + (size_t)ctx->vals_tot * 8 +
               (size_t)ctx->nnz_tot * 8 + (size_t)ctx->xvec_tot * 3 * 8 + (size_t)ctx->ne_tot * ctx->GEO * 8 +
               (size_t)(ctx->mf_F_len + ctx->mf_dinv_len + ctx->mf_upd_len + 2 * (ctx->mf ? ctx->xvec_tot : 0)) * Tsz;
  ctx->budget = budget;
  if (budget > 0 && est > budget) {
    ctx->err = "device footprint " + std::to_string(est) + " B exceeds the budget";
    return TPNS_EBUDGET;
  }
  {
    // every band LU must fit one CTA's shared memory (the panel of NB + kl rows)
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "no CUDA device";
      return TPNS_EDEVICE;
    }
    const size_t need_local = ctx->prec == TPNS_FP64 ? band_lu_smem_bytes<double>(ctx->kl_max_osl)
                                                     : band_lu_smem_bytes<float>(ctx->kl_max_osl);
    if ((!ctx->mf && need_local > (size_t)smem_max) || band_lu_smem_bytes<double>(ctx->kl_max_cf) > (size_t)smem_max) {
      ctx->err = "band width kl = " + std::to_string(std::max(ctx->mf ? 0 : ctx->kl_max_osl, ctx->kl_max_cf)) +
                 " needs more shared memory per CTA than the device has (" + std::to_string(smem_max) +
                 " B); use more subdomains or the FP32 precision";
      return TPNS_EINVAL;
    }
    if (!band_solve_fits_smem<double>(ctx->n_max_cf, ctx->kmax_cf) ||
        !band_solve_fits_smem<double>(ctx->n_max_cp, ctx->kmax_cp)) {
      ctx->err = "coarse system too large for the on-chip coarse solve; use a larger H";
      return TPNS_EINVAL;
    }
  }
  // element arrays
  const int NPE = ctx->NPE, VPE = ctx->VPE, GEO = ctx->GEO, DIM = ctx->dim;
  std::vector<int32_t> h_eprob(ctx->ne_tot), h_e6((size_t)ctx->ne_tot * NPE), h_e3((size_t)ctx->ne_tot * VPE);
  std::vector<int8_t> h_egam(ctx->ne_tot);
  std::vector<double> h_geo((size_t)ctx->ne_tot * GEO);
  std::vector<int32_t> h_gnode(ctx->nn_tot), h_gam(ctx->nn_tot), h_ndof((size_t)ctx->nn_tot * DIM, -1),
      h_nprob(ctx->nn_tot), h_nvidx(ctx->nn_tot);
  std::vector<int8_t> h_nkind(ctx->nn_tot);
  std::vector<int32_t> h_vloc(ctx->nv_tot), h_vdof(ctx->nv_tot, -1);
  // inverse maps of the coarse problems: coarse mesh node -> local node
  std::vector<int32_t> inv_cp = inverse_map(L.cpo.gnode, L.mpH.nn);
  for (int p = 0; p < ctx->nprob; ++p) {
    const Problem& P = *ctx->probs[p];
    const Mesh& m = P.region == 0 ? (P.coarse ? L.mcH : L.mch) : (P.coarse ? L.mpH : L.mph);
    for (int el = 0; el < P.ne; ++el) {
      int64_t ge = ctx->e_off[p] + el;
      h_eprob[ge] = p;
      for (int k = 0; k < NPE; ++k) h_e6[ge * NPE + k] = P.e6[(size_t)NPE * el + k];
      for (int k = 0; k < VPE; ++k) h_e3[ge * VPE + k] = P.e3[(size_t)VPE * el + k];
      h_egam[ge] = P.egam[el];
      if (DIM == 3) {
        // vertices, J^{-1} (row-major: d xi_r / d x_c), |det J|
        const int32_t* tv = &m.tri[4 * (size_t)P.etri[el]];
        double* g = &h_geo[ge * GEO];
        double J[3][3];
        for (int q = 0; q < 4; ++q)
          for (int c = 0; c < 3; ++c) g[3 * q + c] = m.node[3 * (size_t)tv[q] + c];
        for (int c = 0; c < 3; ++c)
          for (int r = 0; r < 3; ++r) J[c][r] = g[3 * (r + 1) + c] - g[c];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double* Ji = g + 12;
        Ji[0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        Ji[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[3] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        Ji[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[6] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        Ji[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        g[21] = std::fabs(det);
        continue;
      }
      const int32_t* tv = &m.tri[3 * (size_t)P.etri[el]];
      double x0 = m.node[2 * tv[0]], y0 = m.node[2 * tv[0] + 1];
      double x1 = m.node[2 * tv[1]], y1 = m.node[2 * tv[1] + 1];
      double x2 = m.node[2 * tv[2]], y2 = m.node[2 * tv[2] + 1];
      double J00 = x1 - x0, J01 = x2 - x0, J10 = y1 - y0, J11 = y2 - y0;
      double det = J00 * J11 - J01 * J10;
      double* g = &h_geo[ge * 11];
      g[0] = x0; g[1] = y0; g[2] = x1; g[3] = y1; g[4] = x2; g[5] = y2;
      g[6] = J11 / det; g[7] = -J01 / det; g[8] = -J10 / det; g[9] = J00 / det;
      g[10] = std::fabs(det);
    }
    for (int l = 0; l < P.nn; ++l) {
      int64_t gn = ctx->n_off[p] + l;
      h_gnode[gn] = P.gnode[l];
      h_nkind[gn] = P.nkind[l];
      int32_t gs = P.gam_src.empty() ? -1 : P.gam_src[l];
      // the coarse porous state is kept in the coarse Darcy problem's local node order
      if (p == CF && gs >= 0) gs = inv_cp[gs];
      h_gam[gn] = gs;
      h_nprob[gn] = p;
      h_nvidx[gn] = P.vidx[l];
      if (P.kind == PK_OSEEN) {
        for (int c = 0; c < DIM; ++c) h_ndof[(size_t)DIM * gn + c] = P.node_dof[(size_t)DIM * l + c];
      } else {
        h_ndof[(size_t)DIM * gn] = P.node_dof[l];
      }
    }
    for (int vv = 0; vv < P.nvl; ++vv) {
      h_vloc[ctx->v_off[p] + vv] = P.vloc[vv];
      if (P.kind == PK_OSEEN) h_vdof[ctx->v_off[p] + vv] = P.vert_dof[vv];
    }
  }
  TRY(upload(ctx, &ctx->d_eprob, h_eprob));
  TRY(upload(ctx, &ctx->d_e6, h_e6));
  TRY(upload(ctx, &ctx->d_e3, h_e3));
  TRY(upload(ctx, &ctx->d_egam, h_egam));
  TRY(upload(ctx, &ctx->d_geo, h_geo));
  TRY(upload(ctx, &ctx->d_gnode, h_gnode));
  TRY(upload(ctx, &ctx->d_nkind, h_nkind));
  TRY(upload(ctx, &ctx->d_gam_src, h_gam));
  TRY(upload(ctx, &ctx->d_node_dof, h_ndof));
  TRY(upload(ctx, &ctx->d_nprob, h_nprob));
  TRY(upload(ctx, &ctx->d_nvidx, h_nvidx));
  TRY(upload(ctx, &ctx->d_vloc, h_vloc));
  TRY(upload(ctx, &ctx->d_vert_dof, h_vdof));
  std::vector<double> h_ref;
  if (DIM == 3) {
    h_ref.resize(sizeof(RefTables3) / sizeof(double));
    std::memcpy(h_ref.data(), &ctx->ref3, sizeof(RefTables3));
  } else {
    h_ref.resize(sizeof(RefTables) / sizeof(double));
    std::memcpy(h_ref.data(), &ctx->ref, sizeof(RefTables));
  }
  TRY(upload(ctx, &ctx->d_ref, h_ref));
  TRY(upload(ctx, &ctx->d_rowptr, h_rowptr));
  TRY(upload(ctx, &ctx->d_colidx, h_colidx));
  TRY(upload(ctx, &ctx->d_rowof, h_rowof));
  TRY(upload(ctx, &ctx->d_sys, ctx->hsys));
  TRY(upload(ctx, &ctx->d_sys_chol, ctx->hsys_chol));
  ctx->flags_stride *= 2;   // panel flags, then per-block progress counters
  TRY(dalloc(ctx, &ctx->d_epoch, 1));
  CK(cudaMemset(ctx->d_epoch, 0, sizeof(int)));
  TRY(dalloc(ctx, &ctx->d_flags, (size_t)ctx->nsys * ctx->flags_stride));
  CK(cudaMemset(ctx->d_flags, 0, (size_t)ctx->nsys * ctx->flags_stride * sizeof(int)));
  TRY(upload(ctx, &ctx->d_chol, ctx->hchol));
  TRY(upload(ctx, &ctx->d_list_osl, ctx->list_osl));
  TRY(upload(ctx, &ctx->d_list_cf, ctx->list_cf));
  TRY(upload(ctx, &ctx->d_list_dl, ctx->list_dl));
  TRY(upload(ctx, &ctx->d_list_cp, ctx->list_cp));
  TRY(upload(ctx, &ctx->d_list_local, ctx->list_local));
  TRY(dalloc(ctx, &ctx->d_vals, ctx->vals_tot));
  TRY(dalloc(ctx, &ctx->d_b, ctx->xvec_tot));
  TRY(dalloc(ctx, &ctx->d_x, ctx->xvec_tot));
  TRY(dalloc(ctx, &ctx->d_xprev, ctx->xvec_tot));
  CK(cudaMemset(ctx->d_xprev, 0, (size_t)ctx->xvec_tot * 8));
  CK(cudaMemset(ctx->d_x, 0, (size_t)ctx->xvec_tot * 8));   // the first step's initial local iterates
  TRY(dalloc(ctx, &ctx->d_r, ctx->xvec_tot));
  TRY(dalloc(ctx, &ctx->d_rel, ctx->nsys));
  TRY(dalloc(ctx, &ctx->d_relprev, ctx->nsys));
  TRY(dalloc(ctx, &ctx->d_done, ctx->nsys));
  TRY(dalloc(ctx, &ctx->d_iters, ctx->nsys));
  CK(cudaMemset(ctx->d_rel, 0, ctx->nsys * sizeof(double)));
  CK(cudaMemset(ctx->d_iters, 0, ctx->nsys * sizeof(int)));
  CK(cudaMemset(ctx->d_done, 0, ctx->nsys * sizeof(int)));
  TRY(dalloc(ctx, &ctx->d_status, ctx->nsys));
  CK(cudaMemset(ctx->d_status, 0, ctx->nsys * sizeof(int)));
  TRY(dalloc(ctx, &ctx->d_ticket, ctx->nsys));
  CK(cudaMemset(ctx->d_ticket, 0, ctx->nsys * sizeof(int)));
  TRY(dalloc(ctx, &ctx->d_partial, (size_t)ctx->nsys * RES_CHUNKS * 2));
  if (ctx->prec == TPNS_FP64) {
    double *b, *d;
    TRY(dalloc(ctx, &b, ctx->band_local_len));
    TRY(dalloc(ctx, &d, ctx->dinv_local_len));
    ctx->d_band_local = b;
    ctx->d_dinv_local = d;
    if (!band_solve_fits_smem<double>(ctx->n_max_band, ctx->kmax_band)) {
      double* v;
      TRY(dalloc(ctx, &v, ctx->xvec_tot));
      ctx->d_vwork = v;
    }
  } else {
    float *b, *d;
    TRY(dalloc(ctx, &b, ctx->band_local_len));
    TRY(dalloc(ctx, &d, ctx->dinv_local_len));
    ctx->d_band_local = b;
    ctx->d_dinv_local = d;
    if (!band_solve_fits_smem<float>(ctx->n_max_band, ctx->kmax_band)) {
      float* v;
      TRY(dalloc(ctx, &v, ctx->xvec_tot));
      ctx->d_vwork = v;
    }
  }
  TRY(upload(ctx, &ctx->d_list_band, ctx->list_band));
  if (ctx->mf) {
    MFSysDev* d_mfsys;
    MFFrontDev* d_fronts;
    int32_t *d_rows, *d_relmap, *d_ok, *d_oi;
    int64_t* d_cp;
    TRY(upload(ctx, &d_mfsys, ctx->h_mfsys));
    TRY(upload(ctx, &d_fronts, h_fronts));
    TRY(upload(ctx, &d_rows, h_mrows));
    if (h_relmap.empty()) h_relmap.push_back(0);
    if (h_origk.empty()) { h_origk.push_back(0); h_origi.push_back(0); }
    TRY(upload(ctx, &d_relmap, h_relmap));
    TRY(upload(ctx, &d_cp, h_colptr));
    TRY(upload(ctx, &d_ok, h_origk));
    TRY(upload(ctx, &d_oi, h_origi));
    ctx->mf_blocks = (int)h_dblk.size();
    if (h_dblk.empty()) h_dblk.push_back(0);
    if (h_big.empty()) h_big.push_back(0);
    TRY(upload(ctx, &ctx->d_mf_big, h_big));
    TRY(upload(ctx, &ctx->d_mf_dblk, h_dblk));
    // scheduling words: task counters and finished-CTA counts at 0, epochs from 1 (the flags
    // start at 0, so no flag of a launch is set before the launch sets it)
    const int nfr = (int)h_fronts.size();
    std::vector<int32_t> sched = {0, 0, 1, 0, 0, 0, 1, 0};
    std::vector<int32_t> flags((size_t)3 * std::max(nfr, 1), 0);
    int32_t *d_sched, *d_flags;
    TRY(upload(ctx, &d_sched, sched));
    TRY(upload(ctx, &d_flags, flags));
    MFLaunch& M = ctx->mfl;
    M.sys = d_mfsys; M.nsys = (int)ctx->h_mfsys.size(); M.fronts = d_fronts; M.nfront = nfr; M.rows = d_rows; M.relmap = d_relmap; M.colptr = d_cp;
    M.orig_k = d_ok; M.orig_ij = d_oi;
    M.vals = nullptr; M.status = nullptr;   // set below once the values and status words exist
    M.sched = d_sched; M.fflag = d_flags; M.sflag = d_flags + nfr;
    const size_t ts = ctx->prec == TPNS_FP64 ? 8 : 4;
    unsigned char *F, *dv, *y, *d, *u;
    TRY(dalloc(ctx, &F, (size_t)std::max<int64_t>(ctx->mf_F_len, 1) * ts));
    TRY(dalloc(ctx, &dv, (size_t)std::max<int64_t>(ctx->mf_dinv_len, 1) * ts));
    TRY(dalloc(ctx, &y, (size_t)ctx->xvec_tot * ts));
    TRY(dalloc(ctx, &d, (size_t)ctx->xvec_tot * ts));
    TRY(dalloc(ctx, &u, (size_t)std::max<int64_t>(ctx->mf_upd_len, 1) * ts));
    ctx->d_mf_F = F; ctx->d_mf_dinv = dv; ctx->d_mf_y = y; ctx->d_mf_d = d; ctx->d_mf_upd = u;
  }
  TRY(dalloc(ctx, &ctx->d_band_coarse, ctx->band_coarse_len));
  TRY(dalloc(ctx, &ctx->d_dinv_coarse, ctx->dinv_coarse_len));
  {
    // factor slabs; entries outside the matrix stay zero for good
    const size_t tsz = ctx->prec == TPNS_FP64 ? 8 : 4;
    unsigned char *ls, *us;
    TRY(dalloc(ctx, &ls, (size_t)ctx->lslab_local_len * tsz));
    TRY(dalloc(ctx, &us, (size_t)ctx->uslab_local_len * tsz));
    CK(cudaMemset(ls, 0, (size_t)ctx->lslab_local_len * tsz));
    CK(cudaMemset(us, 0, (size_t)ctx->uslab_local_len * tsz));
    ctx->d_lslab_local = ls;
    ctx->d_uslab_local = us;
    TRY(dalloc(ctx, &ctx->d_lslab_coarse, ctx->lslab_coarse_len));
    TRY(dalloc(ctx, &ctx->d_uslab_coarse, ctx->uslab_coarse_len));
    CK(cudaMemset(ctx->d_lslab_coarse, 0, (size_t)ctx->lslab_coarse_len * 8));
    CK(cudaMemset(ctx->d_uslab_coarse, 0, (size_t)ctx->uslab_coarse_len * 8));
    if (ctx->prec != TPNS_FP64) {
      TRY(dalloc(ctx, &ctx->d_band_coarse_f, ctx->band_coarse_len));
      TRY(dalloc(ctx, &ctx->d_dinv_coarse_f, ctx->dinv_coarse_len));
      TRY(dalloc(ctx, &ctx->d_lslab_coarse_f, ctx->lslab_coarse_len));
      TRY(dalloc(ctx, &ctx->d_uslab_coarse_f, ctx->uslab_coarse_len));
      CK(cudaMemset(ctx->d_lslab_coarse_f, 0, (size_t)ctx->lslab_coarse_len * 4));
      CK(cudaMemset(ctx->d_uslab_coarse_f, 0, (size_t)ctx->uslab_coarse_len * 4));
    }
  }
  const int SO = ctx->SO, SD = ctx->SD;
  TRY(dalloc(ctx, &ctx->d_Ke, (size_t)(ctx->ne_osl + ctx->ne_cf) * SO * SO));
  TRY(dalloc(ctx, &ctx->d_Re, (size_t)(ctx->ne_osl + ctx->ne_cf) * SO));
  TRY(dalloc(ctx, &ctx->d_ReD, (size_t)(ctx->ne_dl + ctx->ne_cp) * 3 * SD));
  // scatter maps with global offsets
  auto build_map = [&](int p, bool matrix, std::vector<int32_t>& T_, std::vector<int32_t>& S_) {
    const Problem& P = *ctx->probs[p];
    const std::vector<int32_t>& tg = matrix ? P.mtgt : P.rtgt;
    const std::vector<int32_t>& sr = matrix ? P.msrc : P.rsrc;
    if (P.kind == PK_OSEEN) {
      const SysDev& S = ctx->hsys[ctx->sys_first[p]];
      for (size_t k = 0; k < tg.size(); ++k) {
        if (tg[k] < 0) { T_.push_back(-1); S_.push_back(0); continue; }
        T_.push_back((int32_t)((matrix ? S.val_off : S.x_off) + tg[k]));
        S_.push_back((int32_t)(ctx->e_off[p] * (matrix ? SO * SO : SO) + sr[k]));
      }
    } else {
      const int64_t ebase = ctx->e_off[p] - (P.coarse ? ctx->e_off[p] : ctx->eD0);
      for (int f = 0; f < 3; ++f) {
        const SysDev& S = ctx->hsys[ctx->sys_first[p] + f];
        const int per = matrix ? SD * SD : SD;
        for (size_t k = 0; k < tg.size(); ++k) {
          if (tg[k] < 0) { T_.push_back(-1); S_.push_back(0); continue; }
          int el = sr[k] / per, rem = sr[k] % per;
          T_.push_back((int32_t)((matrix ? S.val_off : S.x_off) + tg[k]));
          S_.push_back((int32_t)(((ebase + el) * 3 + f) * per + rem));
        }
      }
    }
  };
  {
    std::vector<int32_t> t1, s1, t2, s2, t3, s3;
    for (int p = 0; p < ctx->nf; ++p) { build_map(p, true, t1, s1); build_map(p, false, t2, s2); }
    for (int p = CF + 1; p < CP; ++p) build_map(p, false, t3, s3);
    ctx->n_mo = (int64_t)t1.size(); ctx->n_ro = (int64_t)t2.size(); ctx->n_rd = (int64_t)t3.size();
    TRY(upload(ctx, &ctx->d_mo_t, t1)); TRY(upload(ctx, &ctx->d_mo_s, s1));
    TRY(upload(ctx, &ctx->d_ro_t, t2)); TRY(upload(ctx, &ctx->d_ro_s, s2));
    TRY(upload(ctx, &ctx->d_rd_t, t3)); TRY(upload(ctx, &ctx->d_rd_s, s3));
    std::vector<int32_t> a1, b1, a2, b2, a3, b3;
    build_map(CF, true, a1, b1);
    build_map(CF, false, a2, b2);
    build_map(CP, false, a3, b3);
    ctx->n_mcf = (int64_t)a1.size(); ctx->n_rcf = (int64_t)a2.size(); ctx->n_rcp = (int64_t)a3.size();
    TRY(upload(ctx, &ctx->d_mcf_t, a1)); TRY(upload(ctx, &ctx->d_mcf_s, b1));
    TRY(upload(ctx, &ctx->d_rcf_t, a2)); TRY(upload(ctx, &ctx->d_rcf_s, b2));
    TRY(upload(ctx, &ctx->d_rcp_t, a3)); TRY(upload(ctx, &ctx->d_rcp_s, b3));
  }
  // fields
  const int nncH = L.mcH.nn, nvcH = L.mcH.nv, nnpH = L.mpH.nn;
  const int nnc = L.mch.nn, nvc = L.mch.nv, nnp = L.mph.nn;
  TRY(dalloc(ctx, &ctx->d_uc_old, (size_t)nncH * DIM));
  TRY(dalloc(ctx, &ctx->d_uc_new, (size_t)nncH * DIM));
  TRY(dalloc(ctx, &ctx->d_pc_new, (size_t)nvcH));
  TRY(dalloc(ctx, &ctx->d_pd_old, (size_t)nnpH * 3));
  TRY(dalloc(ctx, &ctx->d_pd_new, (size_t)nnpH * 3));
  size_t zlen = std::max<size_t>((size_t)nnpH * 3, (size_t)(DIM * L.cfl.nn + L.cfl.nvl));
  TRY(dalloc(ctx, &ctx->d_zero, zlen));
  CK(cudaMemset(ctx->d_zero, 0, zlen * sizeof(double)));
  TRY(dalloc(ctx, &ctx->d_delta, (size_t)(DIM * L.cfl.nn + L.cfl.nvl)));
  TRY(dalloc(ctx, &ctx->d_FW1, (size_t)nnc * DIM));
  TRY(dalloc(ctx, &ctx->d_FW0, (size_t)nnc * DIM));
  TRY(dalloc(ctx, &ctx->d_FP1, (size_t)nvc));
  TRY(dalloc(ctx, &ctx->d_FPD1, (size_t)nnp * 3));
  TRY(dalloc(ctx, &ctx->d_FPD0, (size_t)nnp * 3));
  TRY(dalloc(ctx, &ctx->d_out_u, (size_t)nnc * DIM));
  TRY(dalloc(ctx, &ctx->d_out_p, (size_t)nvc));
  TRY(dalloc(ctx, &ctx->d_out_pd, (size_t)nnp * 3));
  // prolongation tables; the porous coarse index is remapped to the coarse Darcy local order
  std::vector<int32_t> pp2 = L.pp2_idx;
  for (auto& c : pp2) c = inv_cp[c];
  TRY(upload(ctx, &ctx->d_pc2i, L.pc2_idx)); TRY(upload(ctx, &ctx->d_pc2w, L.pc2_w));
  TRY(upload(ctx, &ctx->d_pc1i, L.pc1_idx)); TRY(upload(ctx, &ctx->d_pc1w, L.pc1_w));
  TRY(upload(ctx, &ctx->d_pp2i, pp2)); TRY(upload(ctx, &ctx->d_pp2w, L.pp2_w));
  // glue tables: problem indices of porous locals are shifted in the descriptor array
  std::vector<int32_t> gp_prob = L.gp_prob;
  TRY(upload(ctx, &ctx->d_gc_ptr, L.gc_ptr)); TRY(upload(ctx, &ctx->d_gc_prob, L.gc_prob));
  TRY(upload(ctx, &ctx->d_gc_node, L.gc_node)); TRY(upload(ctx, &ctx->d_gc_w, L.gc_w));
  TRY(upload(ctx, &ctx->d_gp_ptr, L.gp_ptr)); TRY(upload(ctx, &ctx->d_gp_prob, gp_prob));
  TRY(upload(ctx, &ctx->d_gp_node, L.gp_node)); TRY(upload(ctx, &ctx->d_gp_w, L.gp_w));
  TRY(upload(ctx, &ctx->d_gv_ptr, L.gv_ptr)); TRY(upload(ctx, &ctx->d_gv_prob, L.gv_prob));
  TRY(upload(ctx, &ctx->d_gv_vert, L.gv_vert)); TRY(upload(ctx, &ctx->d_gv_w, L.gv_w));
  TRY(dalloc(ctx, &ctx->d_tnow, 1));
  TRY(dalloc(ctx, &ctx->d_step, 1));
  TRY(dalloc(ctx, &ctx->d_newton_done, 1));
  TRY(dalloc(ctx, &ctx->d_newton_iters, 1));
  // local correction state
  std::vector<double*> state(ctx->nprob, nullptr);
  for (int p = 0; p < ctx->nprob; ++p) {
    const Problem& P = *ctx->probs[p];
    if (p == CF || p == CP) continue;
    size_t len = P.kind == PK_OSEEN ? (size_t)(DIM * P.nn + P.nvl) : (size_t)3 * P.nn;
    TRY(dalloc(ctx, &state[p], len));
  }
  // descriptors
  ctx->hprob.assign(ctx->nprob, ProbDev{});
  for (int p = 0; p < ctx->nprob; ++p) {
    const Problem& P = *ctx->probs[p];
    ProbDev& D = ctx->hprob[p];
    D.kind = P.kind; D.coarse = P.coarse; D.dim = DIM; D.ne = P.ne; D.nn = P.nn; D.nvl = P.nvl; D.n = P.n;
    D.e_off = ctx->e_off[p]; D.n_off = ctx->n_off[p]; D.v_off = ctx->v_off[p];
    D.x_off = ctx->hsys[ctx->sys_first[p]].x_off;
    D.fstride = 0;
    if (P.kind == PK_OSEEN && !P.coarse) {
      D.W1 = ctx->d_FW1; D.W0 = ctx->d_FW0; D.P1 = ctx->d_FP1; D.GAM = ctx->d_FPD0;
      D.EN = state[p]; D.EOUT = state[p]; D.XY = nullptr;
    } else if (P.kind == PK_OSEEN) {
      D.W1 = ctx->d_uc_new; D.W0 = ctx->d_uc_old; D.P1 = ctx->d_pc_new; D.GAM = ctx->d_pd_old;
      D.EN = ctx->d_zero; D.EOUT = ctx->d_delta;
    } else if (!P.coarse) {
      D.W1 = ctx->d_FPD1; D.W0 = ctx->d_FPD0; D.P1 = nullptr; D.GAM = ctx->d_FW0;
      D.EN = state[p]; D.EOUT = state[p]; D.fstride = nnp;
    } else {
      D.W1 = ctx->d_zero; D.W0 = ctx->d_zero; D.P1 = nullptr; D.GAM = ctx->d_uc_old;
      D.EN = ctx->d_pd_new; D.EOUT = ctx->d_pd_new; D.fstride = 0;
    }
  }
  // node coordinates of the region meshes
  double *xy_ch, *xy_cH, *xy_ph, *xy_pH;
  TRY(upload(ctx, &xy_ch, L.mch.node)); TRY(upload(ctx, &xy_cH, L.mcH.node));
  TRY(upload(ctx, &xy_ph, L.mph.node)); TRY(upload(ctx, &xy_pH, L.mpH.node));
  for (int p = 0; p < ctx->nprob; ++p) {
    const Problem& P = *ctx->probs[p];
    ctx->hprob[p].XY = P.region == 0 ? (P.coarse ? xy_cH : xy_ch) : (P.coarse ? xy_pH : xy_ph);
  }
  TRY(upload(ctx, &ctx->d_probs, ctx->hprob));
  // initial data: coarse interpolants and e^0 = I_h u0 - I_h I_H u0 (0 on the artificial boundary)
  std::vector<double> uc((size_t)nncH * DIM), pc(nvcH), pdl((size_t)nnpH * 3);
  for (int i = 0; i < nncH; ++i) mms_u_node(ctx, L.mcH, i, 0.0, &uc[(size_t)DIM * i]);
  for (int i = 0; i < nvcH; ++i) pc[i] = mms_p_node(ctx, L.mcH, i, 0.0);
  for (int l = 0; l < nnpH; ++l) {
    int g = L.cpo.gnode[l];
    for (int f = 0; f < 3; ++f) pdl[(size_t)f * nnpH + l] = mms_pd_node(ctx, f, L.mpH, g, 0.0);
  }
  CK(cudaMemcpy(ctx->d_uc_old, uc.data(), uc.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_uc_new, uc.data(), uc.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pc_new, pc.data(), pc.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pd_old, pdl.data(), pdl.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pd_new, pdl.data(), pdl.size() * 8, cudaMemcpyHostToDevice));
  ctx->stats.h2d_bytes += (int64_t)(2 * uc.size() + pc.size() + 2 * pdl.size()) * 8;
  // fine interpolants of the coarse initial data (host, same tables as the device)
  std::vector<double> Iuh((size_t)nnc * DIM, 0.0), Ipdh((size_t)nnp * 3, 0.0);
  for (int i = 0; i < nnc; ++i)
    for (int k = 0; k < NPE; ++k) {
      int c = L.pc2_idx[(size_t)i * NPE + k];
      double w = L.pc2_w[(size_t)i * NPE + k];
      for (int d = 0; d < DIM; ++d) Iuh[(size_t)DIM * i + d] += w * uc[(size_t)DIM * c + d];
    }
  for (int i = 0; i < nnp; ++i)
    for (int k = 0; k < NPE; ++k) {
      int c = pp2[(size_t)i * NPE + k];
      double w = L.pp2_w[(size_t)i * NPE + k];
      for (int f = 0; f < 3; ++f) Ipdh[(size_t)f * nnp + i] += w * pdl[(size_t)f * nnpH + c];
    }
  for (int p = 0; p < ctx->nprob; ++p) {
    if (p == CF || p == CP) continue;
    const Problem& P = *ctx->probs[p];
    std::vector<double> e0;
    if (P.kind == PK_OSEEN) {
      e0.assign((size_t)DIM * P.nn + P.nvl, 0.0);
      for (int l = 0; l < P.nn; ++l) {
        if (P.nkind[l] == 2) continue;
        int g = P.gnode[l];
        double u[3];
        mms_u_node(ctx, L.mch, g, 0.0, u);
        for (int d = 0; d < DIM; ++d) e0[(size_t)DIM * l + d] = u[d] - Iuh[(size_t)DIM * g + d];
      }
    } else {
      e0.assign((size_t)3 * P.nn, 0.0);
      for (int l = 0; l < P.nn; ++l) {
        if (P.nkind[l] == 2) continue;
        int g = P.gnode[l];
        for (int f = 0; f < 3; ++f)
          e0[(size_t)f * P.nn + l] = mms_pd_node(ctx, f, L.mph, g, 0.0) - Ipdh[(size_t)f * nnp + g];
      }
    }
    CK(cudaMemcpy(state[p], e0.data(), e0.size() * 8, cudaMemcpyHostToDevice));
    ctx->stats.h2d_bytes += (int64_t)e0.size() * 8;
  }
  int64_t zero64 = 0;
  CK(cudaMemcpy(ctx->d_step, &zero64, 8, cudaMemcpyHostToDevice));
  // assembly / glue argument blocks
  AsmArgs& A = ctx->asmargs;
  A.probs = ctx->d_probs; A.eprob = ctx->d_eprob; A.geo = ctx->d_geo; A.e6 = ctx->d_e6; A.e3 = ctx->d_e3;
  A.egam = ctx->d_egam; A.gnode = ctx->d_gnode; A.nkind = ctx->d_nkind; A.gam_src = ctx->d_gam_src;
  A.node_dof = ctx->d_node_dof; A.vloc = ctx->d_vloc; A.vert_dof = ctx->d_vert_dof; A.ref = ctx->d_ref;
  A.phys = ctx->phys; A.tnow = ctx->d_tnow; A.dim = DIM;
  GlueArgs& G = ctx->glue;
  G.fluid = ctx->d_probs;
  G.porous = ctx->d_probs + (ctx->nf + 1);
  G.gc_ptr = ctx->d_gc_ptr; G.gc_prob = ctx->d_gc_prob; G.gc_node = ctx->d_gc_node; G.gc_w = ctx->d_gc_w;
  G.gp_ptr = ctx->d_gp_ptr; G.gp_prob = ctx->d_gp_prob; G.gp_node = ctx->d_gp_node; G.gp_w = ctx->d_gp_w;
  G.gv_ptr = ctx->d_gv_ptr; G.gv_prob = ctx->d_gv_prob; G.gv_vert = ctx->d_gv_vert; G.gv_w = ctx->d_gv_w;
  G.FW1 = ctx->d_FW1; G.FP1 = ctx->d_FP1; G.FPD1 = ctx->d_FPD1;
  G.out_u = ctx->d_out_u; G.out_p = ctx->d_out_p; G.out_pd = ctx->d_out_pd;
  G.nnc = nnc; G.nvc = nvc; G.nnp = nnp; G.dim = DIM;
  G.add_coarse = ctx->rank == 0 ? 1 : 0;
  ctx->mfl.vals = ctx->d_vals;
  ctx->mfl.status = ctx->d_status;
  return TPNS_OK;
}

// ------------------------------------------------------------------------------ timing
static cudaEvent_t ev_get(tpns_ctx* ctx) {
  if (ctx->ev_pool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = ctx->ev_pool.back();
  ctx->ev_pool.pop_back();
  return e;
}
static void ph_begin(tpns_ctx* ctx, int id) {
  if (!ctx->timing) return;
  cudaEvent_t e = ev_get(ctx);
  cudaEventRecord(e, ctx->stream);
  ctx->ev_open[id] = e;
}
static void ph_end(tpns_ctx* ctx, int id) {
  if (!ctx->timing || !ctx->ev_open[id]) return;
  cudaEvent_t e = ev_get(ctx);
  cudaEventRecord(e, ctx->stream);
  ctx->ev_pending.push_back({id, {ctx->ev_open[id], e}});
  ctx->ev_open[id] = nullptr;
}
static void ph_collect(tpns_ctx* ctx) {
  for (auto& p : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      ctx->ph_ms[p.first] += ms;
      ctx->ph_n[p.first] += 1;
    }
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
}

// ------------------------------------------------------------------------------ step
static tpns_status prolong_and_glue(tpns_ctx* ctx) {
  const Layout& L = ctx->L;
  cudaStream_t st = ctx->stream;
  CK(launch_prolong(L.mch.nn, L.mch.nv, L.mph.nn, ctx->d_pc2i, ctx->d_pc2w, ctx->d_pc1i, ctx->d_pc1w, ctx->d_pp2i,
                    ctx->d_pp2w, ctx->d_uc_new, ctx->d_uc_old, ctx->d_pc_new, ctx->d_pd_new, ctx->d_pd_old, L.mpH.nn,
                    ctx->d_FW1, ctx->d_FW0, ctx->d_FP1, ctx->d_FPD1, ctx->d_FPD0, L.mph.nn, st, ctx->dim));
  return TPNS_OK;
}

// refinement passes of a coarse Newton correction (FP32 factors): the first residual, then
// up to COARSE_IR_MAX - 1 solve + residual pairs; converged passes exit at once
constexpr int COARSE_IR_MAX = 6;

static tpns_status coarse_step(tpns_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int CF = ctx->nf, CP = ctx->nf + 1 + ctx->np;
  const Layout& L = ctx->L;
  // Step 1(1): coarse Darcy solves (eqs. pFFully, pfFully, pmFully), Cholesky factors fixed
  CK(cudaMemcpyAsync(ctx->d_pd_new, ctx->d_pd_old, (size_t)L.mpH.nn * 3 * 8, cudaMemcpyDeviceToDevice, st));
  double* ReCP = ctx->d_ReD + ctx->ne_dl * 3 * ctx->SD;
  CK(launch_darcy_elem(ctx->asmargs, ctx->e_off[CP], ctx->ne_cp, ReCP, nullptr, st));
  CK(launch_seg_reduce(ctx->d_rcp_t, ctx->d_rcp_s, ctx->n_rcp, ReCP, ctx->d_b, st, nullptr));
  CK(launch_band_solve<double>(ctx->d_sys, ctx->d_list_cp, 3, ctx->n_max_cp, ctx->kmax_cp, ctx->d_lslab_coarse,
                               ctx->d_uslab_coarse, ctx->d_dinv_coarse, ctx->d_b, ctx->d_x, 0, nullptr, ctx->d_status,
                               st, nullptr));
  CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_cp, ctx->nn_cp, ctx->d_x, st, nullptr));
  // Step 1(2): coarse conduit problem (eq. pcFully) by Newton's method
  CK(cudaMemcpyAsync(ctx->d_uc_new, ctx->d_uc_old, (size_t)L.mcH.nn * ctx->dim * 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(ctx->d_newton_done, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_newton_iters, 0, sizeof(int), st));
  const int* skip = ctx->d_newton_done;
  for (int it = 0; it < 12; ++it) {
    CK(launch_oseen_elem(ctx->asmargs, ctx->e_off[CF], ctx->ne_cf, ctx->d_Ke, ctx->d_Re, st, skip));
    CK(launch_seg_reduce(ctx->d_mcf_t, ctx->d_mcf_s, ctx->n_mcf, ctx->d_Ke, ctx->d_vals, st, skip));
    CK(launch_seg_reduce(ctx->d_rcf_t, ctx->d_rcf_s, ctx->n_rcf, ctx->d_Re, ctx->d_b, st, skip));
    if (ctx->prec != TPNS_FP64) {
      // Newton correction from FP32 band factors of the Jacobian, refined against the FP64
      // Jacobian: FP64 arithmetic is scarce on this GPU, FP64 residuals are cheap
      CK(launch_band_fill<float>(ctx->d_sys, ctx->d_list_cf, 1, ctx->d_rowof, ctx->d_colidx, ctx->d_vals,
                                 ctx->d_band_coarse_f, 0, 0, st, skip));
      CK(launch_band_lu<float>(ctx->d_sys, ctx->d_list_cf, 1, ctx->kl_max_cf, ctx->d_band_coarse_f,
                               ctx->d_lslab_coarse_f, ctx->d_uslab_coarse_f, ctx->d_dinv_coarse_f, ctx->d_flags,
                               ctx->flags_stride, ctx->d_epoch, ctx->d_status, st, skip));
      CK(launch_band_dinv<float>(ctx->d_sys, ctx->d_list_cf, 1, ctx->nblk_max_cf, ctx->d_band_coarse_f,
                                 ctx->d_dinv_coarse_f, st, skip));
      const double tol = 1e-13;
      CK(launch_residual(ctx->d_sys, ctx->d_list_cf, 1, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b, ctx->d_x,
                         ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial,
                         ctx->d_ticket, tol, 1, st, skip));
      CK(launch_band_solve<float>(ctx->d_sys, ctx->d_list_cf, 1, ctx->n_max_cf, ctx->kmax_cf, ctx->d_lslab_coarse_f,
                                  ctx->d_uslab_coarse_f, ctx->d_dinv_coarse_f, ctx->d_b, ctx->d_x, 0, nullptr,
                                  ctx->d_status, st, skip));
      for (int r = 0; r < COARSE_IR_MAX; ++r) {
        CK(launch_residual(ctx->d_sys, ctx->d_list_cf, 1, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b,
                           ctx->d_x, ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial,
                           ctx->d_ticket, tol, 0, st, skip));
        if (r + 1 < COARSE_IR_MAX)
          CK(launch_band_solve<float>(ctx->d_sys, ctx->d_list_cf, 1, ctx->n_max_cf, ctx->kmax_cf,
                                      ctx->d_lslab_coarse_f, ctx->d_uslab_coarse_f, ctx->d_dinv_coarse_f, ctx->d_r,
                                      ctx->d_x, 1, ctx->d_done, ctx->d_status, st, skip));
      }
    } else {
      CK(launch_band_fill<double>(ctx->d_sys, ctx->d_list_cf, 1, ctx->d_rowof, ctx->d_colidx, ctx->d_vals,
                                  ctx->d_band_coarse, 0, 0, st, skip));
      CK(launch_band_lu<double>(ctx->d_sys, ctx->d_list_cf, 1, ctx->kl_max_cf, ctx->d_band_coarse,
                                ctx->d_lslab_coarse, ctx->d_uslab_coarse, ctx->d_dinv_coarse, ctx->d_flags,
                                ctx->flags_stride, ctx->d_epoch, ctx->d_status, st, skip));
      CK(launch_band_dinv<double>(ctx->d_sys, ctx->d_list_cf, 1, ctx->nblk_max_cf, ctx->d_band_coarse,
                                  ctx->d_dinv_coarse, st, skip));
      CK(launch_band_solve<double>(ctx->d_sys, ctx->d_list_cf, 1, ctx->n_max_cf, ctx->kmax_cf, ctx->d_lslab_coarse,
                                   ctx->d_uslab_coarse, ctx->d_dinv_coarse, ctx->d_b, ctx->d_x, 0, nullptr,
                                   ctx->d_status, st, skip));
    }
    CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_cf, ctx->nn_cf, ctx->d_x, st, skip));
    CK(launch_newton_update(ctx->d_probs + CF, ctx->d_gnode, ctx->d_vloc, L.cfl.nn, L.cfl.nvl, ctx->d_uc_new,
                            ctx->d_pc_new, ctx->d_newton_done, ctx->d_newton_iters, st));
  }
  return TPNS_OK;
}

template <typename T>
static tpns_status local_step(tpns_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  T* band = reinterpret_cast<T*>(ctx->d_band_local);
  T* dinv = reinterpret_cast<T*>(ctx->d_dinv_local);
  T* vwork = reinterpret_cast<T*>(ctx->d_vwork);
  T* lslab = reinterpret_cast<T*>(ctx->d_lslab_local);
  T* uslab = reinterpret_cast<T*>(ctx->d_uslab_local);
  const int nosl = (int)ctx->list_osl.size(), nloc = (int)ctx->list_local.size();
  // a1: coarse fields on the fine meshes
  ph_begin(ctx, PH_PROLONG);
  TRY(prolong_and_glue(ctx));
  ph_end(ctx, PH_PROLONG);
  // a2-a3: Oseen matrices and right-hand sides of all conduit subdomains
  ph_begin(ctx, PH_ASM_OSEEN);
  CK(launch_oseen_elem(ctx->asmargs, 0, ctx->ne_osl, ctx->d_Ke, ctx->d_Re, st, nullptr));
  ph_end(ctx, PH_ASM_OSEEN);
  ph_begin(ctx, PH_SCATTER);
  CK(launch_seg_reduce(ctx->d_mo_t, ctx->d_mo_s, ctx->n_mo, ctx->d_Ke, ctx->d_vals, st, nullptr));
  CK(launch_seg_reduce(ctx->d_ro_t, ctx->d_ro_s, ctx->n_ro, ctx->d_Re, ctx->d_b, st, nullptr));
  ph_end(ctx, PH_SCATTER);
  // a4: Darcy right-hand sides of all porous subdomains
  ph_begin(ctx, PH_ASM_DARCY);
  CK(launch_darcy_elem(ctx->asmargs, ctx->eD0, ctx->ne_dl, ctx->d_ReD, nullptr, st));
  CK(launch_seg_reduce(ctx->d_rd_t, ctx->d_rd_s, ctx->n_rd, ctx->d_ReD, ctx->d_b, st, nullptr));
  ph_end(ctx, PH_ASM_DARCY);
  // a6: LU of every Oseen system (multifrontal fronts or band)
  T* mfF = reinterpret_cast<T*>(ctx->d_mf_F);
  T* mfD = reinterpret_cast<T*>(ctx->d_mf_dinv);
  if (ctx->mf) {
    ph_begin(ctx, PH_BAND_LU);
    CK(launch_mf_factor<T>(ctx->mfl, 0, ctx->mf_small[0], mfF, mfD, ctx->mf_tc, st));
    for (const auto& lv : ctx->mf_big_levels[0])
      CK(launch_mf_big<T>(ctx->mfl, ctx->d_mf_big + lv[0], lv[1], lv[2], lv[3], mfF, mfD, ctx->mf_tc, st));
    CK(launch_mf_dinv<T>(mfD, ctx->d_mf_dblk, ctx->mf_oseen_blocks, st));
    ph_end(ctx, PH_BAND_LU);
  } else {
    ph_begin(ctx, PH_BAND_FILL);
    CK(launch_band_fill<T>(ctx->d_sys, ctx->d_list_osl, nosl, ctx->d_rowof, ctx->d_colidx, ctx->d_vals, band, 0, 0,
                           st, nullptr));
    ph_end(ctx, PH_BAND_FILL);
    ph_begin(ctx, PH_BAND_LU);
    CK(launch_band_lu<T>(ctx->d_sys, ctx->d_list_osl, nosl, ctx->kl_max_osl, band, lslab, uslab, dinv, ctx->d_flags,
                         ctx->flags_stride, ctx->d_epoch, ctx->d_status, st, nullptr,
                         ctx->prec == TPNS_TF32_IR ? 1 : ctx->prec == TPNS_BF16_IR ? 2 : 0, ctx->lu_cl));
    CK(launch_band_dinv<T>(ctx->d_sys, ctx->d_list_osl, nosl, ctx->nblk_max_osl, band, dinv, st, nullptr));
    ph_end(ctx, PH_BAND_LU);
  }
  const int nband = (int)ctx->list_band.size();
  auto solve_pass = [&]() -> tpns_status {
    CK(launch_band_solve<T>(ctx->d_sys, ctx->d_list_band, nband, ctx->n_max_band, ctx->kmax_band, lslab, uslab, dinv,
                            ctx->d_r, ctx->d_x, 1, ctx->d_done, ctx->d_status, st, nullptr, vwork));
    if (ctx->mf)
      CK(launch_mf_solve<T>(ctx->mfl, mfF, mfD, ctx->d_r, ctx->d_x, 1, ctx->d_done, reinterpret_cast<T*>(ctx->d_mf_y),
                            reinterpret_cast<T*>(ctx->d_mf_d), reinterpret_cast<T*>(ctx->d_mf_upd), ctx->mf_m_max,
                            st));
    return TPNS_OK;
  };
  // a8: solves with FP64-residual iterative refinement
  const bool fp64 = ctx->prec == TPNS_FP64;
  const int maxit = ctx->ir_classic_max > 0 ? ctx->ir_classic_max : fp64 ? 2 : 12;
  const double tol = fp64 ? 1e-14 : 1e-13;
  // the refinement starts from a prediction of the local solutions from the last two steps
  // (2 x^n - x^{n-1}; x^n alone at the second step): the local problems change smoothly in
  // time, so the first residual is already small (and often one refinement pass is saved)
  ph_begin(ctx, PH_RESIDUAL);
  CK(launch_predict(ctx->d_x, ctx->d_xprev, ctx->xvec_tot, ctx->d_step, st));
  CK(launch_residual(ctx->d_sys, ctx->d_list_local, nloc, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b,
                     ctx->d_x, ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial, ctx->d_ticket, tol, 2, st,
                     nullptr));
  ph_end(ctx, PH_RESIDUAL);
  ph_begin(ctx, PH_SOLVE);
  TRY(solve_pass());
  ph_end(ctx, PH_SOLVE);
  for (int it = 0; it < maxit; ++it) {
    ph_begin(ctx, PH_RESIDUAL);
    CK(launch_residual(ctx->d_sys, ctx->d_list_local, nloc, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b,
                       ctx->d_x, ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial, ctx->d_ticket, tol, 0, st,
                       nullptr));
    ph_end(ctx, PH_RESIDUAL);
    if (it + 1 < maxit) {
      ph_begin(ctx, PH_SOLVE);
      TRY(solve_pass());
      ph_end(ctx, PH_SOLVE);
    }
  }
  // a9: new corrections and glue
  ph_begin(ctx, PH_STATE_GLUE);
  CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_fl, ctx->nn_fl, ctx->d_x, st, nullptr));
  CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_pl, ctx->nn_pl, ctx->d_x, st, nullptr));
  CK(launch_glue(ctx->glue, st));
  ph_end(ctx, PH_STATE_GLUE);
  return TPNS_OK;
}

static tpns_status end_step_device(tpns_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const Layout& L = ctx->L;
  ph_begin(ctx, PH_COPIES);
  CK(cudaMemcpyAsync(ctx->d_uc_old, ctx->d_uc_new, (size_t)L.mcH.nn * ctx->dim * 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_pd_old, ctx->d_pd_new, (size_t)L.mpH.nn * 3 * 8, cudaMemcpyDeviceToDevice, st));
  CK(launch_set_time(ctx->d_tnow, ctx->d_step, ctx->dt, 1, st));
  ph_end(ctx, PH_COPIES);
  return TPNS_OK;
}

// Enqueue one time step: Step 1 (unless the coarse state was supplied), Steps 3-4, copies.
static tpns_status enqueue_step(tpns_ctx* ctx, bool coarse) {
  if (coarse) {
    ph_begin(ctx, PH_COARSE);
    TRY(coarse_step(ctx));
    ph_end(ctx, PH_COARSE);
  }
  if (ctx->alg1) {
    // Algorithm 1: the coarse (= fine) solution is the result; the corrections stay zero
    ph_begin(ctx, PH_STATE_GLUE);
    TRY(prolong_and_glue(ctx));
    CK(launch_glue(ctx->glue, ctx->stream));
    ph_end(ctx, PH_STATE_GLUE);
  } else if (ctx->prec == TPNS_FP64) {
    TRY(local_step<double>(ctx));
  } else {
    TRY(local_step<float>(ctx));
  }
  // with GMRES-based refinement the step ends after the host has checked the local systems
  if (ctx->gmres && !ctx->alg1) return TPNS_OK;
  return end_step_device(ctx);
}

// Capture one step into a graph; on failure the caller runs the step eagerly.
static bool capture_step(tpns_ctx* ctx, bool coarse, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int64_t l0 = thread_launch_counter();
  tpns_status s = enqueue_step(ctx, coarse);
  // kernels recorded in the graph run at every replay, not now (counted on this thread only:
  // other threads may launch meanwhile)
  const int64_t recorded = thread_launch_counter() - l0;
  count_launches((int)-recorded);
  (coarse ? ctx->kernels_full : ctx->kernels_local) = recorded;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  bool ok = s == TPNS_OK && e == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    *out = nullptr;
  }
  ctx->err.clear();
  return ok;
}

static tpns_status read_stats(tpns_ctx* ctx) {
  std::vector<int> it(ctx->nsys), stt(ctx->nsys);
  std::vector<double> rel(ctx->nsys);
  int nit = 0;
  CK(cudaStreamSynchronize(ctx->stream));
  ph_collect(ctx);
  CK(cudaMemcpy(it.data(), ctx->d_iters, ctx->nsys * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rel.data(), ctx->d_rel, ctx->nsys * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(stt.data(), ctx->d_status, ctx->nsys * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&nit, ctx->d_newton_iters, sizeof(int), cudaMemcpyDeviceToHost));
  int mx = 0;
  double mr = 0;
  int64_t passes = 0;
  double bytes = 0;
  const double tsz = ctx->prec == TPNS_FP64 ? 8.0 : 4.0;
  for (int s : ctx->list_local) {
    mx = std::max(mx, it[s]);
    mr = std::max(mr, rel[s]);
    // each residual after a solve counts one iteration, so iters = solve passes this step
    const SysDev& S = ctx->hsys[s];
    passes += it[s];
    if (!ctx->mf)
      bytes += (double)it[s] * ((double)S.n * (S.kl + S.ku) * tsz + (double)((S.n + 31) / 32) * 2048.0 * tsz +
                                24.0 * S.n);
  }
  if (ctx->mf)
    for (int q = 0; q < ctx->nprob; ++q) {
      const Problem& P = *ctx->probs[q];
      if (P.coarse) continue;
      const MFSymbolic& M = P.mf;
      double dv = 0;
      for (const MFFront& F : M.fronts) dv += (double)((F.p + MF_NB - 1) / MF_NB) * 2 * MF_NB * MF_NB;
      for (int f = 0; f < (P.kind == PK_OSEEN ? 1 : 3); ++f) {
        const int s = ctx->sys_first[q] + f;
        bytes += (double)it[s] * ((M.factor_entries + dv) * tsz + 24.0 * ctx->hsys[s].n);
      }
    }
  ctx->stats.last_ir_solves = passes;
  ctx->stats.last_solve_bytes = bytes;
  ctx->stats.step = ctx->step;
  ctx->stats.last_ir_iters_max = mx;
  ctx->stats.last_ir_relres_max = mr;
  ctx->stats.last_newton_iters = nit;
  for (int s = 0; s < ctx->nsys; ++s)
    if (stt[s] & 1) {
      ctx->err = "zero or non-finite pivot in system " + std::to_string(s);
      return TPNS_EBREAKDOWN;
    }
  for (int s = 0; s < ctx->nsys; ++s)
    if (stt[s]) {
      ctx->err = "a bounded wait of a device kernel gave up (system " + std::to_string(s) + ")";
      return TPNS_ETIMEOUT;
    }
  if (!(mr <= 1e-9)) {
    ctx->err = "iterative refinement stopped at relative residual " + std::to_string(mr);
    return TPNS_ENOTCONV;
  }
  return TPNS_OK;
}

// GMRES-based refinement of the local systems still above the tolerance after a step's
// classic passes (restarted GMRES, preconditioned by the factors, FP64 vectors), then new
// corrections and glue from the refined solutions.  Eager launches with host checks between
// restart cycles; runs only when needed.
constexpr int GM_KDIM = 10, GM_CYCLES = 4;

template <typename T>
static tpns_status gmres_refine(tpns_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const double tol = ctx->prec == TPNS_FP64 ? 1e-14 : 1e-13;
  const int nloc = (int)ctx->list_local.size();
  const int gstride = (GM_KDIM + 1) * GM_KDIM + (GM_KDIM + 1) + 2 * GM_KDIM;
  std::vector<double> rel(ctx->nsys);
  std::vector<int> skip(ctx->nsys, 1);
  auto pending = [&]() -> int {
    int any = 0;
    std::fill(skip.begin(), skip.end(), 1);
    for (int s : ctx->list_local)
      if (!(rel[s] <= tol)) { skip[s] = 0; any = 1; }
    return any;
  };
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(rel.data(), ctx->d_rel, ctx->nsys * sizeof(double), cudaMemcpyDeviceToHost));
  ctx->stats.last_gmres_outer = 0;
  if (!pending()) return TPNS_OK;
  if (!ctx->gm_V) {
    TRY(dalloc(ctx, &ctx->gm_V, (size_t)(GM_KDIM + 1) * ctx->xvec_tot));
    TRY(dalloc(ctx, &ctx->gm_W, (size_t)ctx->xvec_tot));
    TRY(dalloc(ctx, &ctx->gm_H, (size_t)nloc * gstride));
    TRY(dalloc(ctx, &ctx->gm_skip, (size_t)ctx->nsys));
  }
  T* mfF = reinterpret_cast<T*>(ctx->d_mf_F);
  T* mfD = reinterpret_cast<T*>(ctx->d_mf_dinv);
  T* lslab = reinterpret_cast<T*>(ctx->d_lslab_local);
  T* uslab = reinterpret_cast<T*>(ctx->d_uslab_local);
  T* dinv = reinterpret_cast<T*>(ctx->d_dinv_local);
  T* vwork = reinterpret_cast<T*>(ctx->d_vwork);
  const int nband = (int)ctx->list_band.size();
  // z = M^{-1} w for the pending systems (the factorisation's own solve, overwriting z)
  auto precond = [&](const double* w, double* z) -> tpns_status {
    CK(launch_band_solve<T>(ctx->d_sys, ctx->d_list_band, nband, ctx->n_max_band, ctx->kmax_band, lslab, uslab, dinv,
                            w, z, 0, ctx->gm_skip, ctx->d_status, st, nullptr, vwork));
    if (ctx->mf)
      CK(launch_mf_solve<T>(ctx->mfl, mfF, mfD, w, z, 0, ctx->gm_skip, reinterpret_cast<T*>(ctx->d_mf_y),
                            reinterpret_cast<T*>(ctx->d_mf_d), reinterpret_cast<T*>(ctx->d_mf_upd), ctx->mf_m_max,
                            st));
    return TPNS_OK;
  };
  const int64_t vs = ctx->xvec_tot;
  for (int cyc = 0; cyc < GM_CYCLES; ++cyc) {
    CK(cudaMemcpyAsync(ctx->gm_skip, skip.data(), ctx->nsys * sizeof(int), cudaMemcpyHostToDevice, st));
    // r = b - A x; V[0] = M^{-1} r, normalised
    CK(launch_residual(ctx->d_sys, ctx->d_list_local, nloc, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b,
                       ctx->d_x, ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial,
                       ctx->d_ticket, tol, 2, st, nullptr));
    TRY(precond(ctx->d_r, ctx->gm_V));
    CK(launch_gm_begin(ctx->d_sys, ctx->d_list_local, nloc, ctx->gm_V, vs, ctx->gm_H, gstride, GM_KDIM, ctx->gm_skip,
                       st));
    for (int j = 0; j < GM_KDIM; ++j) {
      CK(launch_spmv(ctx->d_sys, ctx->d_list_local, nloc, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals,
                     ctx->gm_V + (int64_t)j * vs, ctx->gm_W, ctx->gm_skip, st));
      TRY(precond(ctx->gm_W, ctx->gm_V + (int64_t)(j + 1) * vs));
      CK(launch_gm_arnoldi(ctx->d_sys, ctx->d_list_local, nloc, ctx->gm_V, vs, ctx->gm_H, gstride, GM_KDIM, j,
                           ctx->gm_skip, st));
    }
    CK(launch_gm_finish(ctx->d_sys, ctx->d_list_local, nloc, ctx->gm_V, vs, ctx->gm_H, gstride, GM_KDIM, ctx->d_x,
                        ctx->gm_skip, st));
    CK(launch_residual(ctx->d_sys, ctx->d_list_local, nloc, ctx->d_rowptr, ctx->d_colidx, ctx->d_vals, ctx->d_b,
                       ctx->d_x, ctx->d_r, ctx->d_rel, ctx->d_relprev, ctx->d_done, ctx->d_iters, ctx->d_partial,
                       ctx->d_ticket, tol, 2, st, nullptr));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(rel.data(), ctx->d_rel, ctx->nsys * sizeof(double), cudaMemcpyDeviceToHost));
    ctx->stats.last_gmres_outer = cyc + 1;
    if (!pending()) break;
  }
  ctx->stats.gmres_steps += 1;
  // new corrections and glue from the refined local solutions
  CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_fl, ctx->nn_fl, ctx->d_x, st, nullptr));
  CK(launch_state(ctx->asmargs, ctx->d_nprob, ctx->d_nvidx, ctx->nb_pl, ctx->nn_pl, ctx->d_x, st, nullptr));
  CK(launch_glue(ctx->glue, st));
  return TPNS_OK;
}

static tpns_status run_steps(tpns_ctx* ctx, int nsteps, bool from_traj) {
  for (int s = 0; s < nsteps; ++s) {
    if (from_traj) {
      int64_t k = ctx->step - ctx->traj_base;
      if (k < 0 || k + 1 >= (int64_t)ctx->traj.size()) {
        ctx->err = "no stored coarse state for this step";
        return TPNS_EINVAL;
      }
      const Layout& L = ctx->L;
      size_t nu = (size_t)L.mcH.nn * ctx->dim, npc = L.mcH.nv, npd = (size_t)L.mpH.nn * 3;
      cudaStream_t st = ctx->stream;
      CK(cudaMemcpyAsync(ctx->d_uc_old, ctx->traj[k], nu * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ctx->d_pd_old, ctx->traj[k] + nu + npc, npd * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ctx->d_uc_new, ctx->traj[k + 1], nu * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ctx->d_pc_new, ctx->traj[k + 1] + nu, npc * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ctx->d_pd_new, ctx->traj[k + 1] + nu + npc, npd * 8, cudaMemcpyDeviceToDevice, st));
    }
    bool graph = ctx->use_graph && !ctx->timing;
    if (graph) {
      cudaGraphExec_t& ex = from_traj ? ctx->g_local : ctx->g_full;
      if (!ex && !capture_step(ctx, !from_traj, &ex)) {
        ctx->use_graph = false;
        graph = false;
      }
      if (graph) {
        CK(cudaGraphLaunch(ex, ctx->stream));
        count_launches((int)(from_traj ? ctx->kernels_local : ctx->kernels_full));
      }
    }
    if (!graph) TRY(enqueue_step(ctx, !from_traj));
    if (ctx->gmres && !ctx->alg1) {
      TRY(ctx->prec == TPNS_FP64 ? gmres_refine<double>(ctx) : gmres_refine<float>(ctx));
      TRY(end_step_device(ctx));
    }
    ctx->step += 1;
  }
  return read_stats(ctx);
}

// Launch tuning of the Oseen band LU on the context's own systems: where both 8- and 16-CTA
// clusters can be placed, factor the (zeroed) bands with each twice and keep the faster;
// the work of an unpivoted band LU does not depend on the values.  Runs before the Darcy
// factors exist; it writes only in-band slab entries (those outside the matrix stay zero) and
// the status words are reset afterwards.
template <typename T>
static tpns_status tune_lu(tpns_ctx* ctx) {
  const int nosl = (int)ctx->list_osl.size();
  ctx->lu_cl = LU_CLUSTER;
  if (nosl == 0) return TPNS_OK;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nosl * 2 * LU_CLUSTER > nsm) return TPNS_OK;   // only 8-CTA clusters fit at once
  cudaStream_t st = ctx->stream;
  T* band = reinterpret_cast<T*>(ctx->d_band_local);
  const int tc = ctx->prec == TPNS_TF32_IR ? 1 : ctx->prec == TPNS_BF16_IR ? 2 : 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int pick = LU_CLUSTER;
  for (int cl : {LU_CLUSTER, 2 * LU_CLUSTER}) {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaMemsetAsync(band, 0, (size_t)ctx->band_local_len * sizeof(T), st));
      CK(cudaEventRecord(e0, st));
      CK(launch_band_lu<T>(ctx->d_sys, ctx->d_list_osl, nosl, ctx->kl_max_osl, band,
                           reinterpret_cast<T*>(ctx->d_lslab_local), reinterpret_cast<T*>(ctx->d_uslab_local),
                           reinterpret_cast<T*>(ctx->d_dinv_local), ctx->d_flags, ctx->flags_stride, ctx->d_epoch,
                           ctx->d_status, st, nullptr, tc, cl));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
    }
    if (ms < best) {
      best = ms;
      pick = cl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->lu_cl = pick;
  CK(cudaMemsetAsync(ctx->d_status, 0, ctx->nsys * sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  return TPNS_OK;
}

static tpns_status setup_factors(tpns_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int CP = ctx->nf + 1 + ctx->np;
  // Darcy element matrices (run once) -> CSR values -> band Cholesky
  const int64_t neD = ctx->ne_dl + ctx->ne_cp;
  double* KeD = nullptr;
  const int SD = ctx->SD;
  TRY(dalloc(ctx, &KeD, (size_t)neD * 3 * SD * SD));
  std::vector<int32_t> t1, s1, t2, s2;
  for (int p = ctx->nf + 1; p <= CP; ++p) {
    const Problem& P = *ctx->probs[p];
    const int64_t ebase = ctx->e_off[p] - ctx->eD0;
    for (int f = 0; f < 3; ++f) {
      const SysDev& S = ctx->hsys[ctx->sys_first[p] + f];
      for (size_t k = 0; k < P.mtgt.size(); ++k) {
        if (P.mtgt[k] < 0) { t1.push_back(-1); s1.push_back(0); continue; }
        int el = P.msrc[k] / (SD * SD), rem = P.msrc[k] % (SD * SD);
        t1.push_back((int32_t)(S.val_off + P.mtgt[k]));
        s1.push_back((int32_t)(((ebase + el) * 3 + f) * SD * SD + rem));
      }
    }
  }
  int32_t *dt1, *ds1;
  TRY(upload(ctx, &dt1, t1));
  TRY(upload(ctx, &ds1, s1));
  CK(launch_set_time(ctx->d_tnow, ctx->d_step, ctx->dt, 0, st));
  CK(launch_darcy_elem(ctx->asmargs, ctx->eD0, neD, nullptr, KeD, st));
  CK(launch_seg_reduce(dt1, ds1, (int64_t)t1.size(), KeD, ctx->d_vals, st, nullptr));
  const int ndl = (int)ctx->list_dl.size();
  // one-time band Cholesky of every Darcy system, rewritten as unit-L / U factors
  {
    double* cband;
    TRY(dalloc(ctx, &cband, ctx->band_chol_coarse_len));
    CK(launch_band_fill<double>(ctx->d_sys_chol, ctx->d_list_cp, 3, ctx->d_rowof, ctx->d_colidx, ctx->d_vals, cband, 1,
                                0, st, nullptr));
    CK(launch_band_chol<double>(ctx->d_sys_chol, ctx->d_list_cp, 3, cband, ctx->d_status, st));
    CK(launch_chol_to_lu<double>(ctx->d_sys_chol, ctx->d_sys, ctx->d_list_cp, 3, cband, ctx->d_band_coarse, st));
    CK(launch_band_to_slab<double>(ctx->d_sys, ctx->d_list_cp, 3, ctx->d_band_coarse, ctx->d_lslab_coarse,
                                   ctx->d_uslab_coarse, st));
    CK(launch_band_dinv<double>(ctx->d_sys, ctx->d_list_cp, 3, ctx->nblk_max_cp, ctx->d_band_coarse,
                                ctx->d_dinv_coarse, st, nullptr));
  }
  if (ctx->mf) {
    // the local Darcy systems: multifrontal LU once (their matrices do not change)
    const int nd = ctx->mfl.nfront - ctx->mf_oseen_fronts;
    const int nb = ctx->mf_blocks - ctx->mf_oseen_blocks;
    (void)nd;
    if (ctx->prec == TPNS_FP64) {
      CK(launch_mf_factor<double>(ctx->mfl, ctx->mf_oseen_fronts, ctx->mf_small[1], reinterpret_cast<double*>(ctx->d_mf_F),
                                  reinterpret_cast<double*>(ctx->d_mf_dinv), 0, st));
      for (const auto& lv : ctx->mf_big_levels[1])
        CK(launch_mf_big<double>(ctx->mfl, ctx->d_mf_big + lv[0], lv[1], lv[2], lv[3], reinterpret_cast<double*>(ctx->d_mf_F),
                                 reinterpret_cast<double*>(ctx->d_mf_dinv), 0, st));
      CK(launch_mf_dinv<double>(reinterpret_cast<double*>(ctx->d_mf_dinv), ctx->d_mf_dblk + ctx->mf_oseen_blocks, nb,
                                st));
    } else {
      CK(launch_mf_factor<float>(ctx->mfl, ctx->mf_oseen_fronts, ctx->mf_small[1], reinterpret_cast<float*>(ctx->d_mf_F),
                                 reinterpret_cast<float*>(ctx->d_mf_dinv), ctx->mf_tc, st));
      for (const auto& lv : ctx->mf_big_levels[1])
        CK(launch_mf_big<float>(ctx->mfl, ctx->d_mf_big + lv[0], lv[1], lv[2], lv[3], reinterpret_cast<float*>(ctx->d_mf_F),
                                reinterpret_cast<float*>(ctx->d_mf_dinv), ctx->mf_tc, st));
      CK(launch_mf_dinv<float>(reinterpret_cast<float*>(ctx->d_mf_dinv), ctx->d_mf_dblk + ctx->mf_oseen_blocks, nb,
                               st));
    }
  } else if (ctx->prec == TPNS_FP64) {
    double* band = reinterpret_cast<double*>(ctx->d_band_local);
    double* dinv = reinterpret_cast<double*>(ctx->d_dinv_local);
    double* cband;
    TRY(dalloc(ctx, &cband, ctx->band_chol_local_len));
    CK(launch_band_fill<double>(ctx->d_sys_chol, ctx->d_list_dl, ndl, ctx->d_rowof, ctx->d_colidx, ctx->d_vals, cband, 1,
                                0, st, nullptr));
    CK(launch_band_chol<double>(ctx->d_sys_chol, ctx->d_list_dl, ndl, cband, ctx->d_status, st));
    CK(launch_chol_to_lu<double>(ctx->d_sys_chol, ctx->d_sys, ctx->d_list_dl, ndl, cband, band, st));
    CK(launch_band_to_slab<double>(ctx->d_sys, ctx->d_list_dl, ndl, band, (double*)ctx->d_lslab_local,
                                   (double*)ctx->d_uslab_local, st));
    CK(launch_band_dinv<double>(ctx->d_sys, ctx->d_list_dl, ndl, ctx->nblk_max_dl, band, dinv, st, nullptr));
  } else {
    float* band = reinterpret_cast<float*>(ctx->d_band_local);
    float* dinv = reinterpret_cast<float*>(ctx->d_dinv_local);
    float* cband;
    TRY(dalloc(ctx, &cband, ctx->band_chol_local_len));
    CK(launch_band_fill<float>(ctx->d_sys_chol, ctx->d_list_dl, ndl, ctx->d_rowof, ctx->d_colidx, ctx->d_vals, cband, 1,
                               0, st, nullptr));
    CK(launch_band_chol<float>(ctx->d_sys_chol, ctx->d_list_dl, ndl, cband, ctx->d_status, st));
    CK(launch_chol_to_lu<float>(ctx->d_sys_chol, ctx->d_sys, ctx->d_list_dl, ndl, cband, band, st));
    CK(launch_band_to_slab<float>(ctx->d_sys, ctx->d_list_dl, ndl, band, (float*)ctx->d_lslab_local,
                                  (float*)ctx->d_uslab_local, st));
    CK(launch_band_dinv<float>(ctx->d_sys, ctx->d_list_dl, ndl, ctx->nblk_max_dl, band, dinv, st, nullptr));
  }
  // initial glued fields
  TRY(prolong_and_glue(ctx));
  CK(launch_glue(ctx->glue, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int> stt(ctx->nsys);
  CK(cudaMemcpy(stt.data(), ctx->d_status, ctx->nsys * sizeof(int), cudaMemcpyDeviceToHost));
  for (int s = 0; s < ctx->nsys; ++s)
    if (stt[s] & 1) {
      ctx->err = "Darcy factorisation: zero, non-positive or non-finite pivot in system " + std::to_string(s);
      return TPNS_EBREAKDOWN;
    }
  for (int s = 0; s < ctx->nsys; ++s)
    if (stt[s]) {
      ctx->err = "a bounded wait of a device kernel gave up (system " + std::to_string(s) + ")";
      return TPNS_ETIMEOUT;
    }
  return TPNS_OK;
}

// ------------------------------------------------------------------------------ standalone solve
__global__ void csr_rowof_kernel(const int32_t* __restrict__ rowptr, int n, int32_t* __restrict__ rowof) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) rowof[k] = i;
}

// Run the band solver on one system whose descriptors and scratch live at caller-chosen
// device addresses (`sysd`: SysDev, `listd`: int 0, `vecs`: r, rel, relprev, done, iters,
// status, flags).  The band and dinv buffers must hold n * (kl + ku + 1) and
// ceil(n / 32) * 2048 elements of T; vwork holds n elements of T (the solve vector of a
// system too large for shared memory).  Every return, failed or not, leaves the stream
// synchronised, so no work of the call still touches the scratch afterwards.
template <typename T>
static tpns_status band_solve_run(int n, int kl, int ku, const int32_t* rowptr, const int32_t* colidx,
                                  const double* vals, const double* b, double* x, cudaStream_t st, SysDev* sysd,
                                  int* listd, int32_t* rowof, T* band, T* dinv, T* lslab, T* uslab, T* vwork,
                                  double* r, double* rel, double* relprev, int* done, int* iters, int* status,
                                  int* flags, int epoch, double* relres_out, std::string& err) {
  // the residual's partial sums follow the vector r; its ticket follows the status word
  double* partial = r + n + 2;
  int* ticket = status + 1;
#define CKS(call)                                                           \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      cudaStreamSynchronize(st);                                            \
      return TPNS_EDEVICE;                                                  \
    }                                                                       \
  } while (0)
  int nnz = 0;
  CKS(cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  SysDev S{};
  S.n = n; S.kl = kl; S.ku = ku; S.ldab = kl + ku + 1;
  S.band_off = 0; S.rp_off = 0; S.nnz_off = 0; S.nnz = nnz; S.val_off = 0; S.x_off = 0; S.dinv_off = 0;
  S.lslab_off = 0; S.uslab_off = 0;
  const int nblk = (n + LU_NB - 1) / LU_NB;
  CKS(cudaMemsetAsync(lslab, 0, (size_t)nblk * LU_NB * kl * sizeof(T), st));
  CKS(cudaMemsetAsync(uslab, 0, (size_t)nblk * LU_NB * ku * sizeof(T), st));
  CKS(cudaMemsetAsync(flags, 0, sizeof(int) * 2 * (size_t)nblk, st));
  const int zero = 0;
  CKS(cudaMemcpyAsync(sysd, &S, sizeof(SysDev), cudaMemcpyHostToDevice, st));
  CKS(cudaMemcpyAsync(listd, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
  CKS(cudaMemsetAsync(status, 0, sizeof(int), st));
  count_launches(1);
  csr_rowof_kernel<<<(n + 255) / 256, 256, 0, st>>>(rowptr, n, rowof);
  CKS(cudaGetLastError());
  CKS(launch_band_fill<T>(sysd, listd, 1, rowof, colidx, vals, band, 0, 0, st, nullptr));
  int* epoch_dev = flags + 2 * nblk;
  CKS(cudaMemcpyAsync(epoch_dev, &epoch, sizeof(int), cudaMemcpyHostToDevice, st));
  CKS(launch_band_lu<T>(sysd, listd, 1, kl, band, lslab, uslab, dinv, flags, 2 * nblk, epoch_dev, status, st, nullptr));
  CKS(launch_band_dinv<T>(sysd, listd, 1, nblk, band, dinv, st, nullptr));
  const bool fp64 = sizeof(T) == 8;
  const int maxit = 12;
  const double tol = fp64 ? 1e-14 : 1e-13;
  const int kmax = std::max(kl, ku);
  CKS(cudaMemsetAsync(ticket, 0, sizeof(int), st));
  CKS(launch_residual(sysd, listd, 1, rowptr, colidx, vals, b, x, r, rel, relprev, done, iters, partial, ticket, tol, 1,
                      st, nullptr));
  CKS(launch_band_solve<T>(sysd, listd, 1, n, kmax, lslab, uslab, dinv, b, x, 0, nullptr, status, st, nullptr,
                           vwork));
  for (int it = 0; it < maxit; ++it) {
    CKS(launch_residual(sysd, listd, 1, rowptr, colidx, vals, b, x, r, rel, relprev, done, iters, partial, ticket, tol,
                        0, st, nullptr));
    if (it + 1 < maxit)
      CKS(launch_band_solve<T>(sysd, listd, 1, n, kmax, lslab, uslab, dinv, r, x, 1, done, status, st, nullptr,
                               vwork));
  }
  int hst = 0;
  double hrel = 0;
  CKS(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(&hrel, rel, sizeof(double), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (relres_out) *relres_out = hrel;
  if (hst & 1) {
    err = "zero or non-finite pivot";
    return TPNS_EBREAKDOWN;
  }
  if (hst) {
    err = "a bounded wait of a device kernel gave up";
    return TPNS_ETIMEOUT;
  }
  if (!(hrel <= 1e-9)) {
    err = "iterative refinement stopped at relative residual " + std::to_string(hrel);
    return TPNS_ENOTCONV;
  }
  return TPNS_OK;
#undef CKS
}

// epoch tag of the standalone solves' panel flags (shared by all host threads)
static std::atomic<int> g_solve_epoch{0};

static tpns_status band_solve_check(int32_t n, int32_t kl, int32_t ku, const int32_t* rowptr, const int32_t* colidx,
                                    const double* vals, const double* b, double* x, tpns_precision precision) {
  if (n <= 0 || kl < 0 || ku < 1 || kl + LU_NB > 512 || ku + LU_NB > 512 || !rowptr || !colidx || !vals || !b ||
      !x) {
    g_err = "invalid band solve arguments";
    return TPNS_EINVAL;
  }
  if (precision != TPNS_FP64 && precision != TPNS_FP32_IR) {
    g_err = "precision not available in this build";
    return TPNS_EINVAL;
  }
  return TPNS_OK;
}

// ------------------------------------------------------------------------------ no-allocation solve
// Scratch of tpns_band_solve_noalloc, shared by all its calls on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TPNS_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device (looked up once per device).
static tpns_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    g_err = "no current CUDA device";
    return TPNS_EDEVICE;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return TPNS_EDEVICE;
    }
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TPNS_OK;
}

// ------------------------------------------------------------------------------ ABI
extern "C" {

tpns_status tpns_create(const tpns_mesh_desc* mesh, const tpns_params* params, const tpns_partition_desc* part,
                        const tpns_data_desc* data, double dt, tpns_precision precision, size_t hbm_budget_bytes,
                        void* cuda_stream, tpns_ctx** out) {
  return tpns_create_ex(mesh, params, part, data, dt, precision, hbm_budget_bytes, cuda_stream, nullptr, out);
}

static bool read_options(const tpns_options* o, tpns_options& opt) {
  opt = tpns_options{};
  if (o) opt = *o;
  if (opt.local_factor != TPNS_FACTOR_MULTIFRONTAL && opt.local_factor != TPNS_FACTOR_BAND) return false;
  if (opt.mf_leaf < 0 || opt.mf_ctas < 0) return false;
  if (opt.nranks < 0 || (opt.nranks > 0 && (opt.rank < 0 || opt.rank >= opt.nranks))) return false;
  if (opt.nranks == 0) opt.nranks = 1;
  if (opt.algorithm == 0) opt.algorithm = 3;
  if (opt.algorithm != 1 && opt.algorithm != 3) return false;
  if (opt.refinement < 0 || opt.refinement > 1 || opt.ir_classic_max < 0 || opt.ir_classic_max > 64) return false;
  if (opt.mf_leaf == 0) opt.mf_leaf = 96;
  if (opt.mf_leaf < 8) return false;
  if (opt.mf_big_m == 0) opt.mf_big_m = 256;
  if (opt.mf_big_m > 0 && opt.mf_big_m < 128) return false;
  return true;
}

tpns_status tpns_create_ex(const tpns_mesh_desc* mesh, const tpns_params* params, const tpns_partition_desc* part,
                           const tpns_data_desc* data, double dt, tpns_precision precision, size_t hbm_budget_bytes,
                           void* cuda_stream, const tpns_options* options, tpns_ctx** out) {
  g_err.clear();
  const auto t_create = std::chrono::steady_clock::now();
  tpns_options opt;
  if (!read_options(options, opt)) { g_err = "invalid options"; return TPNS_EINVAL; }
  if (opt.local_factor == TPNS_FACTOR_MULTIFRONTAL && precision == TPNS_BF16_IR) {
    g_err = "TPNS_BF16_IR is available with the band factorisation only";
    return TPNS_EINVAL;
  }
  if (!out) { g_err = "out is NULL"; return TPNS_EINVAL; }
  *out = nullptr;
  if (!mesh || !params || !part || !data) { g_err = "NULL argument"; return TPNS_EINVAL; }
  if (!(dt > 0)) { g_err = "dt must be positive"; return TPNS_EINVAL; }
  if (precision != TPNS_FP64 && precision != TPNS_FP32_IR && precision != TPNS_TF32_IR &&
      precision != TPNS_BF16_IR) {
    g_err = "precision not available in this build";
    return TPNS_EINVAL;
  }
  if (!(params->nu > 0 && params->eta > 0 && params->rho > 0 && params->mu > 0 && params->alpha >= 0 &&
        params->k[0] > 0 && params->k[1] > 0 && params->k[2] > 0 && params->phiC[0] > 0 && params->phiC[1] > 0 &&
        params->phiC[2] > 0 && params->sigma >= 0 && params->sigma_star >= 0)) {
    g_err = "invalid physical parameters";
    return TPNS_EINVAL;
  }
  if (mesh->dim == 3 ? (data->mms_id != 0 && data->mms_id != 2 && data->mms_id != 4)
                     : (data->mms_id != 0 && data->mms_id != 1 && data->mms_id != 3)) {
    g_err = "unknown mms_id for this mesh dimension";
    return TPNS_EINVAL;
  }
  tpns_mesh_desc md1 = *mesh;
  tpns_partition_desc pd1 = *part;
  if (opt.algorithm == 1) {
    // Algorithm 1: the same decoupled steps on the fine grid itself (H = h, no subdomains)
    const int r = mesh->fine_rows_from_gamma[0];
    for (int c = 0; c < mesh->ny_coarse && c < TPNS_MAX_COARSE_ROWS; ++c)
      if (mesh->fine_rows_from_gamma[c] != r) { g_err = "Algorithm 1 needs uniform fine rows"; return TPNS_EINVAL; }
    if ((int64_t)mesh->ny_coarse * r > TPNS_MAX_COARSE_ROWS || opt.nranks > 1) {
      g_err = "Algorithm 1: more fine rows than TPNS_MAX_COARSE_ROWS, or a rank split";
      return TPNS_EINVAL;
    }
    md1.nx_coarse = mesh->nx_coarse * mesh->fine_per_coarse_x;
    md1.fine_per_coarse_x = 1;
    md1.ny_coarse = mesh->ny_coarse * r;
    for (int c = 0; c < md1.ny_coarse; ++c) md1.fine_rows_from_gamma[c] = 1;
    pd1.nsub_x = pd1.nsub_y = 1;
    pd1.overlap = 0;
    mesh = &md1;
    part = &pd1;
  }
  tpns_ctx* ctx = new (std::nothrow) tpns_ctx();
  if (!ctx) { g_err = "host allocation failed"; return TPNS_ENOMEM; }
  ctx->alg1 = opt.algorithm == 1;
  ctx->gmres = opt.refinement == 1;
  ctx->ir_classic_max = opt.ir_classic_max;
  cudaGetDevice(&ctx->device);
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!ctx->stream) {
    // a blocking stream keeps the ordering with the legacy default stream and can be captured
    if (cudaStreamCreate(&ctx->stream) == cudaSuccess) ctx->own_stream = true;
    else ctx->stream = nullptr;
  }
  ctx->prec = precision;
  ctx->dt = dt;
  ctx->mf = opt.local_factor == TPNS_FACTOR_MULTIFRONTAL;
  ctx->mf_leaf = opt.mf_leaf;
  ctx->mf_big_m = opt.mf_big_m;
  ctx->mf_tc = precision != TPNS_FP64 && !opt.mf_cuda_cores;
  ctx->rank = opt.rank;
  ctx->nranks = opt.nranks;
  ctx->mfl.grid_cap = opt.mf_ctas;
  Phys& P = ctx->phys;
  P.nu = params->nu; P.eta = params->eta; P.rho = params->rho; P.mu = params->mu; P.alpha = params->alpha;
  P.sigma = params->sigma; P.sigma_star = params->sigma_star;
  for (int i = 0; i < 3; ++i) { P.phiC[i] = params->phiC[i]; P.k[i] = params->k[i]; }
  P.dt = dt;
  P.mms = data->mms_id;
  tpns_status s = build_ctx(ctx, *mesh, *part, hbm_budget_bytes);
  // the tuning runs before the Darcy factors are formed: it overwrites the local bands, and
  // setup_factors then writes the Darcy bands, slabs and inverses from scratch
  if (s == TPNS_OK && !ctx->mf) s = ctx->prec == TPNS_FP64 ? tune_lu<double>(ctx) : tune_lu<float>(ctx);
  if (s == TPNS_OK) s = setup_factors(ctx);
  if (s != TPNS_OK) {
    g_err = ctx->err;
    tpns_destroy(ctx);
    return s;
  }
  ctx->stats.n_fine_dofs = (int64_t)ctx->L.mch.nn * ctx->dim + ctx->L.mch.nv + (int64_t)ctx->L.mph.nn * 3;
  ctx->stats.n_local_systems = (int64_t)ctx->list_local.size();
  ctx->stats.device_bytes = (int64_t)ctx->bytes;
  ctx->stats.band_lu_flops = ctx->lu_flops_step;
  ctx->stats.lu_cluster_ctas = ctx->mf ? 0 : ctx->lu_cl;
  for (int q = 0; q < ctx->nf; ++q) {
    const Problem& P = *ctx->probs[q];
    ctx->stats.oseen_unknowns += P.n;
    ctx->stats.oseen_nnz += (int64_t)P.colidx.size();
    ctx->stats.oseen_elements += P.ne;
    if (ctx->mf) ctx->stats.mf_fronts += (int64_t)P.mf.fronts.size();
    if (!ctx->mf) {
      for (int j = 0; j < P.n; ++j) {
        const double l = std::min(P.kl, P.n - 1 - j), u = std::min(P.ku, P.n - 1 - j);
        ctx->stats.factor_entries += 1 + l + u;
      }
    }
  }
  if (ctx->mf) ctx->stats.factor_entries = ctx->mf_factor_entries;
  for (int q = ctx->nf + 1; q < ctx->nf + 1 + ctx->np; ++q) {
    ctx->stats.darcy_unknowns += 3 * (int64_t)ctx->probs[q]->n;
    ctx->stats.darcy_elements += ctx->probs[q]->ne;
  }
  ctx->stats.create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_create).count();
  *out = ctx;
  return TPNS_OK;
}

tpns_status tpns_layout_create(const tpns_mesh_desc* mesh, const tpns_partition_desc* part, tpns_ctx** out) {
  return tpns_layout_create_ex(mesh, part, nullptr, out);
}

tpns_status tpns_layout_create_ex(const tpns_mesh_desc* mesh, const tpns_partition_desc* part,
                                  const tpns_options* options, tpns_ctx** out) {
  g_err.clear();
  if (!out || !mesh || !part) { g_err = "NULL argument"; return TPNS_EINVAL; }
  *out = nullptr;
  tpns_options opt;
  if (!read_options(options, opt)) { g_err = "invalid options"; return TPNS_EINVAL; }
  tpns_ctx* ctx = new (std::nothrow) tpns_ctx();
  if (!ctx) return TPNS_ENOMEM;
  ctx->host_only = true;
  ctx->mf = opt.local_factor == TPNS_FACTOR_MULTIFRONTAL;
  ctx->mf_leaf = opt.mf_leaf;
  ctx->rank = opt.rank;
  ctx->nranks = opt.nranks;
  std::string msg = build_layout(*mesh, *part, ctx->L, ctx->mf ? ctx->mf_leaf : 0, ctx->rank, ctx->nranks);
  if (!msg.empty()) {
    g_err = msg;
    delete ctx;
    return TPNS_EINVAL;
  }
  ctx->nf = (int)ctx->L.fluid.size();
  ctx->np = (int)ctx->L.porous.size();
  *out = ctx;
  return TPNS_OK;
}

tpns_status tpns_band_solve(int32_t n, int32_t kl, int32_t ku, const int32_t* rowptr, const int32_t* colidx,
                            const double* vals, const double* b, double* x, tpns_precision precision,
                            void* cuda_stream, double* relres_out) {
  g_err.clear();
  tpns_status s = band_solve_check(n, kl, ku, rowptr, colidx, vals, b, x, precision);
  if (s != TPNS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t tsz = precision == TPNS_FP64 ? 8 : 4;
  const int nblk = (n + LU_NB - 1) / LU_NB;
  int nnz = 0;
  if (cudaMemcpy(&nnz, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    g_err = "cannot read rowptr";
    return TPNS_EDEVICE;
  }
  std::vector<void*> mem;
  auto get = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) return nullptr;
    mem.push_back(p);
    return p;
  };
  void* band = get((size_t)n * (kl + ku + 1) * tsz);
  void* dinv = get((size_t)nblk * 2 * LU_NB * LU_NB * tsz);
  void* lsl = get((size_t)nblk * LU_NB * kl * tsz);
  void* usl = get((size_t)nblk * LU_NB * ku * tsz);
  void* vw = get((size_t)n * tsz);
  SysDev* sysd = (SysDev*)get(sizeof(SysDev));
  int* ints = (int*)get(sizeof(int) * (6 + 2 * (size_t)nblk));
  int32_t* rowof = (int32_t*)get(sizeof(int32_t) * (size_t)std::max(nnz, 1));
  double* dbl = (double*)get(sizeof(double) * ((size_t)n + 2 + 2 * RES_CHUNKS));
  tpns_status out;
  if (!band || !dinv || !lsl || !usl || !vw || !sysd || !ints || !rowof || !dbl) {
    g_err = "cudaMalloc failed";
    out = TPNS_ENOMEM;
  } else {
    cudaMemsetAsync(ints, 0, sizeof(int) * (6 + 2 * (size_t)nblk), st);
    int* listd = ints;
    int* done = ints + 1;
    int* iters = ints + 2;
    int* status = ints + 3;
    int* flags = ints + 5;
    double* r = dbl;
    double* rel = dbl + n;
    double* relprev = dbl + n + 1;
    const int epoch = ++g_solve_epoch;
    if (precision == TPNS_FP64)
      out = band_solve_run<double>(n, kl, ku, rowptr, colidx, vals, b, x, st, sysd, listd, rowof, (double*)band,
                                   (double*)dinv, (double*)lsl, (double*)usl, (double*)vw, r, rel, relprev, done,
                                   iters, status, flags, epoch, relres_out, g_err);
    else
      out = band_solve_run<float>(n, kl, ku, rowptr, colidx, vals, b, x, st, sysd, listd, rowof, (float*)band,
                                  (float*)dinv, (float*)lsl, (float*)usl, (float*)vw, r, rel, relprev, done, iters,
                                  status, flags, epoch, relres_out, g_err);
  }
  cudaStreamSynchronize(st);
  for (void* p : mem) cudaFree(p);
  return out;
}

tpns_status tpns_band_solve_noalloc(int32_t n, int32_t kl, int32_t ku, const int32_t* rowptr, const int32_t* colidx,
                                    const double* vals, const double* b, double* x, tpns_precision precision,
                                    void* cuda_stream, double* relres_out) {
  g_err.clear();
  tpns_status s = band_solve_check(n, kl, ku, rowptr, colidx, vals, b, x, precision);
  if (s != TPNS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != TPNS_OK) return s;
  int nnz = 0;
  if (cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    g_err = "cannot read rowptr";
    return TPNS_EDEVICE;
  }
  // carve the scratch: every piece 256-byte aligned
  const size_t tsz = precision == TPNS_FP64 ? 8 : 4;
  const int nblk = (n + LU_NB - 1) / LU_NB;
  size_t off = 0;
  auto take = [&](size_t bytes) -> size_t {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_band = take((size_t)n * (kl + ku + 1) * tsz);
  const size_t o_dinv = take((size_t)nblk * 2 * LU_NB * LU_NB * tsz);
  const size_t o_lsl = take((size_t)nblk * LU_NB * kl * tsz);
  const size_t o_usl = take((size_t)nblk * LU_NB * ku * tsz);
  const size_t o_vw = take((size_t)n * tsz);
  const size_t o_sys = take(sizeof(SysDev));
  const size_t o_ints = take(sizeof(int) * (6 + 2 * (size_t)nblk));
  const size_t o_rowof = take(sizeof(int32_t) * (size_t)std::max(nnz, 1));
  const size_t o_dbl = take(sizeof(double) * ((size_t)n + 2 + 2 * RES_CHUNKS));
  if (nnz < 0 || off > (size_t)TPNS_NOALLOC_SCRATCH_BYTES) {
    g_err = "system needs " + std::to_string(off) + " bytes of scratch; tpns_band_solve_noalloc has " +
            std::to_string((size_t)TPNS_NOALLOC_SCRATCH_BYTES);
    return TPNS_EINVAL;
  }
  int* ints = reinterpret_cast<int*>(base + o_ints);
  // done, iters, status and the panel flags / block counters must start at zero
  if (cudaMemsetAsync(ints, 0, sizeof(int) * (6 + 2 * (size_t)nblk), st) != cudaSuccess) {
    g_err = "cudaMemsetAsync failed";
    return TPNS_EDEVICE;
  }
  double* dbl = reinterpret_cast<double*>(base + o_dbl);
  const int epoch = ++g_solve_epoch;
  if (precision == TPNS_FP64)
    return band_solve_run<double>(n, kl, ku, rowptr, colidx, vals, b, x, st, reinterpret_cast<SysDev*>(base + o_sys),
                                  ints, reinterpret_cast<int32_t*>(base + o_rowof),
                                  reinterpret_cast<double*>(base + o_band), reinterpret_cast<double*>(base + o_dinv),
                                  reinterpret_cast<double*>(base + o_lsl), reinterpret_cast<double*>(base + o_usl),
                                  reinterpret_cast<double*>(base + o_vw), dbl, dbl + n, dbl + n + 1, ints + 1, ints + 2, ints + 3, ints + 5, epoch, relres_out,
                                  g_err);
  return band_solve_run<float>(n, kl, ku, rowptr, colidx, vals, b, x, st, reinterpret_cast<SysDev*>(base + o_sys), ints,
                               reinterpret_cast<int32_t*>(base + o_rowof), reinterpret_cast<float*>(base + o_band),
                               reinterpret_cast<float*>(base + o_dinv), reinterpret_cast<float*>(base + o_lsl),
                               reinterpret_cast<float*>(base + o_usl), reinterpret_cast<float*>(base + o_vw), dbl,
                               dbl + n, dbl + n + 1, ints + 1, ints + 2,
                               ints + 3, ints + 5, epoch, relres_out, g_err);
}

tpns_status tpns_debug_fronts(const tpns_ctx* ctx, int32_t j, int32_t what, int32_t* dst, size_t* n) {
  if (!ctx || !n || !ctx->mf || j < 0 || j >= (int)ctx->L.fluid.size()) return TPNS_EINVAL;
  const MFSymbolic& M = ctx->L.fluid[j].mf;
  std::vector<int32_t> v;
  switch (what) {
    case 0: v = {(int32_t)M.fronts.size(), M.nlevels}; break;
    case 1:
      for (const MFFront& F : M.fronts) {
        const int32_t r[7] = {F.m, F.p, F.level, F.parent, F.nchild, F.child[0], F.child[1]};
        v.insert(v.end(), r, r + 7);
      }
      break;
    case 2: for (const MFFront& F : M.fronts) v.insert(v.end(), F.rows.begin(), F.rows.end()); break;
    case 3: for (const MFFront& F : M.fronts) v.insert(v.end(), F.relmap.begin(), F.relmap.end()); break;
    case 4: for (const MFFront& F : M.fronts) v.insert(v.end(), F.col_ptr.begin(), F.col_ptr.end()); break;
    case 5: for (const MFFront& F : M.fronts) v.insert(v.end(), F.orig_k.begin(), F.orig_k.end()); break;
    case 6: for (const MFFront& F : M.fronts) v.insert(v.end(), F.orig_i.begin(), F.orig_i.end()); break;
    case 7: for (const MFFront& F : M.fronts) v.insert(v.end(), F.col_child.begin(), F.col_child.end()); break;
    case 8: v = M.order; break;
    default: return TPNS_EINVAL;
  }
  if (dst) {
    if (*n < v.size()) return TPNS_EINVAL;
    std::copy(v.begin(), v.end(), dst);
  }
  *n = v.size();
  return TPNS_OK;
}

tpns_status tpns_debug_values(tpns_ctx* ctx, int32_t j, int32_t field, double* vals, double* rhs) {
  if (!ctx || ctx->host_only) return TPNS_EINVAL;
  int p;
  if (j >= 0 && j < ctx->nf) p = j;
  else if (j >= ctx->nf && j < ctx->nf + ctx->np) p = j + 1;   // skip the coarse conduit problem
  else return TPNS_EINVAL;
  const Problem& P = *ctx->probs[p];
  const int f = P.kind == PK_OSEEN ? 0 : field;
  if (f < 0 || f > 2) return TPNS_EINVAL;
  const SysDev& S = ctx->hsys[ctx->sys_first[p] + f];
  CK(cudaStreamSynchronize(ctx->stream));
  if (vals) CK(cudaMemcpy(vals, ctx->d_vals + S.val_off, S.nnz * sizeof(double), cudaMemcpyDeviceToHost));
  if (rhs) CK(cudaMemcpy(rhs, ctx->d_b + S.x_off, S.n * sizeof(double), cudaMemcpyDeviceToHost));
  return TPNS_OK;
}

tpns_status tpns_step(tpns_ctx* ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0 || ctx->host_only) return TPNS_EINVAL;
  ctx->err.clear();
  ctx->traj_base = -1000000000;
  return run_steps(ctx, nsteps, false);
}

tpns_status tpns_coarse_precompute(tpns_ctx* ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0 || ctx->host_only) return TPNS_EINVAL;
  ctx->err.clear();
  const Layout& L = ctx->L;
  size_t nu = (size_t)L.mcH.nn * ctx->dim, npc = L.mcH.nv, npd = (size_t)L.mpH.nn * 3;
  size_t len = nu + npc + npd;
  for (double* p : ctx->traj) cudaFree(p), ctx->bytes -= len * 8;
  for (double* p : ctx->traj) {
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), (void*)p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
  }
  ctx->traj.clear();
  if (ctx->budget > 0 && ctx->bytes + (size_t)(nsteps + 1) * len * 8 > ctx->budget) {
    ctx->err = "coarse trajectory of " + std::to_string(nsteps) + " steps exceeds the budget";
    return TPNS_EBUDGET;
  }
  cudaStream_t st = ctx->stream;
  // save the current coarse state, then march the coarse problem alone
  std::vector<double> keep_uc(nu), keep_pc(npc), keep_pd(npd);
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(keep_uc.data(), ctx->d_uc_old, nu * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(keep_pc.data(), ctx->d_pc_new, npc * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(keep_pd.data(), ctx->d_pd_old, npd * 8, cudaMemcpyDeviceToHost));
  int64_t step0 = ctx->step;
  for (int k = 0; k <= nsteps; ++k) {
    double* slot;
    TRY(dalloc(ctx, &slot, len));
    ctx->traj.push_back(slot);
    if (k > 0) {
      TRY(coarse_step(ctx));
      CK(cudaMemcpyAsync(slot, ctx->d_uc_new, nu * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(slot + nu, ctx->d_pc_new, npc * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(slot + nu + npc, ctx->d_pd_new, npd * 8, cudaMemcpyDeviceToDevice, st));
      TRY(end_step_device(ctx));
      ctx->step += 1;
    } else {
      CK(cudaMemcpyAsync(slot, ctx->d_uc_old, nu * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(slot + nu, ctx->d_pc_new, npc * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(slot + nu + npc, ctx->d_pd_old, npd * 8, cudaMemcpyDeviceToDevice, st));
    }
  }
  CK(cudaStreamSynchronize(st));
  // rewind the clock and the coarse state
  CK(cudaMemcpy(ctx->d_uc_old, keep_uc.data(), nu * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_uc_new, keep_uc.data(), nu * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pc_new, keep_pc.data(), npc * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pd_old, keep_pd.data(), npd * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_pd_new, keep_pd.data(), npd * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_step, &step0, 8, cudaMemcpyHostToDevice));
  ctx->step = step0;
  ctx->traj_base = (int)step0;
  return TPNS_OK;
}

tpns_status tpns_local_step(tpns_ctx* ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0 || ctx->host_only) return TPNS_EINVAL;
  ctx->err.clear();
  cudaStream_t st = ctx->stream;
  CK(launch_set_time(ctx->d_tnow, ctx->d_step, ctx->dt, 0, st));
  return run_steps(ctx, nsteps, true);
}

tpns_status tpns_num_dofs(const tpns_ctx* ctx, int32_t field, size_t* n) {
  if (!ctx || !n) return TPNS_EINVAL;
  const Layout& L = ctx->L;
  if (ctx->L.dim == 3) {
    if (field >= 0 && field <= 2) *n = (size_t)L.mch.nn;
    else if (field == 3) *n = (size_t)L.mch.nv;
    else if (field >= 4 && field <= 6) *n = (size_t)L.mph.nn;
    else return TPNS_EINVAL;
    return TPNS_OK;
  }
  switch (field) {
    case 0: case 1: *n = (size_t)L.mch.nn; return TPNS_OK;
    case 2: *n = (size_t)L.mch.nv; return TPNS_OK;
    case 3: case 4: case 5: *n = (size_t)L.mph.nn; return TPNS_OK;
    default: return TPNS_EINVAL;
  }
}

tpns_status tpns_get_field(tpns_ctx* ctx, int32_t field, double* dst, size_t n, int32_t dst_on_device) {
  if (!ctx || !dst || ctx->host_only) return TPNS_EINVAL;
  size_t need = 0;
  if (tpns_num_dofs(ctx, field, &need) != TPNS_OK || n < need) {
    ctx->err = "destination too small or bad field";
    return TPNS_EINVAL;
  }
  cudaStream_t st = ctx->stream;
  const Layout& L = ctx->L;
  CK(cudaStreamSynchronize(st));
  const int D = ctx->dim;
  if (field < D) {
    // strided component of the interleaved velocity
    std::vector<double> tmp((size_t)L.mch.nn * D);
    CK(cudaMemcpy(tmp.data(), ctx->d_out_u, tmp.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<double> comp(L.mch.nn);
    for (int i = 0; i < L.mch.nn; ++i) comp[i] = tmp[(size_t)D * i + field];
    CK(cudaMemcpy(dst, comp.data(), need * 8, dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    return TPNS_OK;
  }
  const double* src = field == D ? ctx->d_out_p : ctx->d_out_pd + (size_t)(field - D - 1) * L.mph.nn;
  CK(cudaMemcpyAsync(dst, src, need * 8, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return TPNS_OK;
}

tpns_status tpns_get_stats(tpns_ctx* ctx, tpns_stats* out) {
  if (!ctx || !out) return TPNS_EINVAL;
  ctx->stats.device_bytes = (int64_t)ctx->bytes;
  *out = ctx->stats;
  return TPNS_OK;
}

tpns_status tpns_batch_step(tpns_ctx** ctxs, int32_t n) {
  if (!ctxs || n < 0) return TPNS_EINVAL;
  g_err.clear();
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || ctxs[i]->host_only || ctxs[i]->device != ctxs[0]->device) {
      g_err = "batch contexts must be device contexts of one device";
      return TPNS_EINVAL;
    }
  // enqueue one step of every context first (each on its own stream, so that their kernels
  // run side by side), then collect the status words
  for (int i = 0; i < n; ++i) {
    tpns_ctx* ctx = ctxs[i];
    ctx->err.clear();
    ctx->traj_base = -1000000000;
    if (!ctx->ev_s0 && (cudaEventCreate(&ctx->ev_s0) != cudaSuccess || cudaEventCreate(&ctx->ev_s1) != cudaSuccess)) {
      g_err = ctx->err = "cudaEventCreate failed";
      return TPNS_EDEVICE;
    }
    // the capture of a first step records no work, so the step's start is marked after it
    bool graph = ctx->use_graph && !ctx->timing;
    if (graph && !ctx->g_full && !capture_step(ctx, true, &ctx->g_full)) {
      ctx->use_graph = false;
      graph = false;
    }
    if (cudaEventRecord(ctx->ev_s0, ctx->stream) != cudaSuccess) {
      g_err = ctx->err = "cudaEventRecord failed";
      return TPNS_EDEVICE;
    }
    if (graph) {
      if (cudaGraphLaunch(ctx->g_full, ctx->stream) != cudaSuccess) {
        g_err = ctx->err = "cudaGraphLaunch failed";
        return TPNS_EDEVICE;
      }
      count_launches((int)ctx->kernels_full);
    } else {
      tpns_status s = enqueue_step(ctx, true);
      if (s != TPNS_OK) {
        g_err = ctx->err;
        return s;
      }
    }
    if (cudaEventRecord(ctx->ev_s1, ctx->stream) != cudaSuccess) {
      g_err = ctx->err = "cudaEventRecord failed";
      return TPNS_EDEVICE;
    }
    ctx->step += 1;
  }
  tpns_status worst = TPNS_OK;
  for (int i = 0; i < n; ++i) {
    tpns_ctx* ctx = ctxs[i];
    tpns_status s = TPNS_OK;
    if (ctx->gmres && !ctx->alg1) {
      // the refinement check and the end of the step of a context with GMRES-based refinement
      s = ctx->prec == TPNS_FP64 ? gmres_refine<double>(ctx) : gmres_refine<float>(ctx);
      if (s == TPNS_OK) s = end_step_device(ctx);
    }
    if (s == TPNS_OK) s = read_stats(ctxs[i]);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctxs[i]->ev_s0, ctxs[i]->ev_s1) == cudaSuccess) ctxs[i]->stats.last_step_ms = ms;
    if (s != TPNS_OK && worst == TPNS_OK) {
      worst = s;
      g_err = ctxs[i]->err;
    }
  }
  return worst;
}

tpns_status tpns_set_timing(tpns_ctx* ctx, int32_t on) {
  if (!ctx || ctx->host_only) return TPNS_EINVAL;
  ctx->timing = on != 0;
  for (int i = 0; i < PH_COUNT; ++i) { ctx->ph_ms[i] = 0; ctx->ph_n[i] = 0; }
  return TPNS_OK;
}

tpns_status tpns_get_timings(const tpns_ctx* ctx, double* ms, int64_t* count, int32_t n) {
  if (!ctx || n < 0) return TPNS_EINVAL;
  for (int i = 0; i < n && i < PH_COUNT; ++i) {
    if (ms) ms[i] = ctx->ph_ms[i];
    if (count) count[i] = ctx->ph_n[i];
  }
  return TPNS_OK;
}

int64_t tpns_launch_count(void) { return tpns::launch_counter(); }

const char* tpns_last_error(const tpns_ctx* ctx) {
  if (!ctx) return g_err.c_str();
  return ctx->err.c_str();
}

void tpns_destroy(tpns_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->g_full) cudaGraphExecDestroy(ctx->g_full);
  if (ctx->g_local) cudaGraphExecDestroy(ctx->g_local);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  for (void* p : ctx->allocs) cudaFree(p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->ev_s0) cudaEventDestroy(ctx->ev_s0);
  if (ctx->ev_s1) cudaEventDestroy(ctx->ev_s1);
  for (auto& p : ctx->ev_pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
  for (double* p : ctx->traj) {
    (void)p;
  }
  delete ctx;
}

tpns_status tpns_debug_mesh(const tpns_ctx* ctx, int32_t what, void* dst, size_t* n) {
  if (!ctx || !n) return TPNS_EINVAL;
  const Layout& L = ctx->L;
  const Mesh* m = (what == 0 || what == 2) ? &L.mch : &L.mph;
  if (what == 0 || what == 1) {
    *n = m->node.size();
    if (dst) std::memcpy(dst, m->node.data(), m->node.size() * sizeof(double));
    return TPNS_OK;
  }
  if (what == 2 || what == 3) {
    *n = m->tri6.size();
    if (dst) std::memcpy(dst, m->tri6.data(), m->tri6.size() * sizeof(int32_t));
    return TPNS_OK;
  }
  return TPNS_EINVAL;
}

tpns_status tpns_debug_system(const tpns_ctx* ctx, int32_t j, int32_t* n_unknowns, int32_t* unknown_node,
                              int32_t* unknown_comp, int64_t* nnz, int32_t* rowptr, int32_t* colidx, int32_t* kl,
                              int32_t* ku) {
  if (!ctx) return TPNS_EINVAL;
  // local systems in order: conduit subdomains, then porous subdomains (one pattern each)
  const Problem* P = nullptr;
  if (j >= 0 && j < ctx->nf) P = &ctx->L.fluid[j];
  else if (j >= ctx->nf && j < ctx->nf + ctx->np) P = &ctx->L.porous[j - ctx->nf];
  else return TPNS_EINVAL;
  if (n_unknowns) *n_unknowns = P->n;
  if (nnz) *nnz = (int64_t)P->colidx.size();
  if (kl) *kl = P->kl;
  if (ku) *ku = P->ku;
  if (unknown_node)
    for (int d = 0; d < P->n; ++d) unknown_node[d] = P->gnode[P->dof_node[d]];
  if (unknown_comp)
    for (int d = 0; d < P->n; ++d) unknown_comp[d] = P->dof_comp[d];
  if (rowptr) std::memcpy(rowptr, P->rowptr.data(), P->rowptr.size() * sizeof(int32_t));
  if (colidx) std::memcpy(colidx, P->colidx.data(), P->colidx.size() * sizeof(int32_t));
  return TPNS_OK;
}

}  // extern "C"
