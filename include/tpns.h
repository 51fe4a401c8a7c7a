/*
 * tpns.h -- C ABI of the GB300 library for the local parallel two-grid finite element
 * method for the transient triple-porosity Navier-Stokes model (Algorithm 3, Sec. 5).
 *
 * The library advances, on one CUDA device, the 2D problem of Sec. 2 on the fluid
 * region [0,1]x[1,2] over the porous region [0,1]x[0,1] (interface Gamma: y = 1):
 *   Step 1  coarse decoupled solves on T_H (eqs. pFFully, pfFully, pmFully, pcFully),
 *   Step 2  overlapping subdomains Omega_j built at create time,
 *   Step 3  local fine corrections on every Omega_j (eqs. pFlocalFully, pflocalFully,
 *           pmlocalFully, uclocalFully): Oseen saddle-point systems factorised every step,
 *           Darcy SPD systems factorised once,
 *   Step 4  correction of data: glued global fine fields.
 * Elements: P2-P1 Taylor-Hood in the conduit, P2 for the three Darcy pressures.
 *
 * Conventions
 *   - All pointers are host pointers unless an argument says otherwise.
 *   - The library copies every input at create time and owns all device state of a
 *     context; outputs go to caller buffers.
 *   - Errors are returned as tpns_status; no exception crosses the ABI.  A context whose
 *     call failed keeps a message readable with tpns_last_error().
 *   - A context is bound to the device that was current at tpns_create and to the CUDA
 *     stream given there; every call enqueues on that stream.  With a NULL stream the
 *     context creates its own blocking stream (ordered with the legacy default stream).
 *   - A time step is captured once into a CUDA graph and replayed (all its loops have fixed
 *     trip counts; convergence is decided on the device); while per-phase timing is on
 *     (tpns_set_timing) steps are launched kernel by kernel instead.
 *   - Field ids: 0 = u_x, 1 = u_y (conduit velocity, P2 nodes), 2 = p (conduit pressure,
 *     vertices), 3 = p_F (macro-fracture), 4 = p_f (micro-fracture), 5 = p_m (matrix), the
 *     last three on the P2 nodes of the porous mesh.  Global fine numbering: vertex
 *     (i, j) -> i + (nx+1) j, then one node per edge, edges sorted by (min, max) vertex id.
 */
#ifndef TPNS_H
#define TPNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPNS_OK = 0,
  TPNS_EINVAL = 1,     /* invalid argument (null pointer, bad size, inconsistent layout) */
  TPNS_ENOMEM = 2,     /* device or host allocation failed */
  TPNS_ENOTCONV = 3,   /* iterative refinement or Newton did not reach its tolerance */
  TPNS_EDEVICE = 4,    /* a CUDA call failed; see tpns_last_error */
  TPNS_ETIMEOUT = 5,   /* a bounded device wait gave up */
  TPNS_EBUDGET = 6,    /* the device footprint exceeds the caller's HBM budget */
  TPNS_EBREAKDOWN = 7  /* a pivot of an unpivoted factorisation was zero or not finite */
} tpns_status;

/* Precision of the local factorisations and triangular solves.  Residuals of the
 * iterative refinement, assembly, the coarse solve and the glue are always FP64. */
typedef enum {
  TPNS_FP64 = 0,       /* FP64 band LU / Cholesky */
  TPNS_FP32_IR = 1,    /* FP32 factors (FP32 FMA), FP64-residual iterative refinement */
  TPNS_TF32_IR = 2,    /* FP32 factors whose trailing (bulk) updates run on the tensor cores:
                          mma.sync TF32 with each operand split in two TF32 parts
                          (hi*hi + hi*lo + lo*hi, FP32 accumulation); tpns_create only */
  TPNS_BF16_IR = 3     /* FP32 factors whose trailing (bulk) updates run on the tensor cores in
                          plain BF16 (mma.sync, each operand rounded once, FP32 accumulation);
                          the refinement must win back BF16-level factor error and may stop
                          with TPNS_ENOTCONV; tpns_create only */
} tpns_precision;

#define TPNS_MAX_COARSE_ROWS 64

/* Mesh of both regions (Sec. 6 Example 1 geometry).  Coarse mesh: nx_coarse columns of
 * width 1/nx_coarse, ny_coarse rows of height 1/ny_coarse per region.  Fine mesh (nested
 * grid lines): every coarse column is split into fine_per_coarse_x equal columns; coarse
 * row c, counted from Gamma outwards in both regions, is split into
 * fine_rows_from_gamma[c] equal rows. */
typedef struct {
  int32_t nx_coarse;
  int32_t ny_coarse;
  int32_t fine_per_coarse_x;
  int32_t fine_rows_from_gamma[TPNS_MAX_COARSE_ROWS];
} tpns_mesh_desc;

/* Physical parameters of Sec. 2 (order of Darcy arrays: F, f, m). */
typedef struct {
  double nu, eta, rho, mu, alpha, sigma, sigma_star;
  double phiC[3];      /* phi_i C_i */
  double k[3];         /* permeabilities */
} tpns_params;

/* Algorithm 3 Step 2: nsub_x x nsub_y boxes D_j per region aligned with coarse lines,
 * enlarged by `overlap` fine layers on sides inside the region. */
typedef struct {
  int32_t nsub_x, nsub_y;
  int32_t overlap;
} tpns_partition_desc;

/* Data of the run: manufactured solution id (1 = 2D trigonometric field, 3 = steady
 * polynomial patch field, 0 = zero data); forcing, boundary and interface data are derived
 * from it. */
typedef struct {
  int32_t mms_id;
} tpns_data_desc;

typedef struct {
  int64_t step;                   /* steps taken */
  int32_t last_ir_iters_max;      /* max IR iterations over local systems, last step */
  int32_t last_newton_iters;      /* coarse Newton iterations, last step */
  double last_ir_relres_max;      /* max ||b - A x|| / ||b|| over local systems, last step */
  int64_t n_fine_dofs;            /* all global fine dofs of all fields */
  int64_t n_local_systems;        /* Oseen + Darcy local systems per step */
  int64_t device_bytes;           /* device footprint of the context */
  double band_lu_flops;           /* algorithmic flops of one step's Oseen band LUs */
  int64_t h2d_bytes;              /* bytes copied host -> device by tpns_create */
  int64_t last_ir_solves;         /* band solve passes over all local systems, last step */
  double last_solve_bytes;        /* algorithmic bytes of those passes: per pass and system
                                     n (kl + ku) s + ceil(n / 32) 2048 s + 24 n, s = factor
                                     element size (factor slabs, diagonal-block inverses, FP64
                                     right-hand side read and solution read + write) */
  double last_step_ms;            /* device time of the context's last step in tpns_batch_step,
                                     from the step's start on its stream to its end (with the
                                     other contexts of the batch running beside it) */
  int64_t lu_cluster_ctas;        /* CTAs per cluster of the Oseen band LU: 8, or 16 where all
                                     clusters fit the device and tpns_create measured 16 faster
                                     on the context's own systems */
} tpns_stats;

typedef struct tpns_ctx tpns_ctx;

/* Build meshes, subdomains, sparsity, scatter maps and band orderings on the host, upload
 * them, factor the time-invariant Darcy blocks and set the initial state (nodal
 * interpolation of the data at t = 0).  `cuda_stream` is a cudaStream_t (NULL = a private
 * blocking stream the context creates and destroys).  hbm_budget_bytes (0 = no limit) caps
 * the context's device footprint: a lower-bound estimate is checked before any allocation,
 * then every allocation (including later ones of tpns_coarse_precompute) is checked against
 * the cap; the first one that would pass it fails the call with TPNS_EBUDGET and whatever the
 * call allocated is released.  On success *out owns the context; release it with
 * tpns_destroy. */
tpns_status tpns_create(const tpns_mesh_desc* mesh, const tpns_params* params,
                        const tpns_partition_desc* part, const tpns_data_desc* data,
                        double dt, tpns_precision precision, size_t hbm_budget_bytes,
                        void* cuda_stream, tpns_ctx** out);

/* Advance nsteps time steps (Algorithm 3 Steps 1, 3, 4 each step), enqueued on the
 * context's stream; returns after the work is enqueued and the step's status word read
 * back (one device-to-host copy of a few bytes per call). */
tpns_status tpns_step(tpns_ctx* ctx, int32_t nsteps);

/* Run Step 1 (coarse decoupled solves) for the next nsteps steps ahead and keep the coarse
 * states on the device, so that tpns_local_step can run Steps 3-4 alone.  Fails with
 * TPNS_EBUDGET, before any work, if the nsteps + 1 stored states would pass the context's
 * HBM budget. */
tpns_status tpns_coarse_precompute(tpns_ctx* ctx, int32_t nsteps);

/* Advance nsteps steps using coarse states stored by tpns_coarse_precompute: the
 * per-step local hot path (prolongation, assembly, factorisation, solves and refinement,
 * glue) only.  Fails with TPNS_EINVAL if fewer coarse states are stored. */
tpns_status tpns_local_step(tpns_ctx* ctx, int32_t nsteps);

/* Number of global fine values of a field (see field ids above). */
tpns_status tpns_num_dofs(const tpns_ctx* ctx, int32_t field, size_t* n);

/* Copy the glued global fine field into dst (n values, FP64).  dst_on_device != 0: dst is
 * a device pointer on the context's device (copied on the context's stream, then the
 * stream is synchronised). */
tpns_status tpns_get_field(tpns_ctx* ctx, int32_t field, double* dst, size_t n,
                           int32_t dst_on_device);

/* Counters of the last step and sizes of the context. */
tpns_status tpns_get_stats(tpns_ctx* ctx, tpns_stats* out);

/* Serving: one time step of each of n contexts.  The steps of all contexts are enqueued
 * first, each on its context's stream (graph replays), so that their assembly, factorisation,
 * solves and glue kernels run side by side on the device; then every context's status is
 * collected.  All contexts must live on the same device.  Returns the first failure
 * (message in tpns_last_error(NULL)); the other contexts still advanced. */
tpns_status tpns_batch_step(tpns_ctx** ctxs, int32_t n);

/* Per-phase device time, measured with CUDA events recorded on the context's stream
 * around each phase of a step while timing is on (tpns_set_timing(ctx, 1) also clears
 * the totals).  Phase ids: 0 coarse solves (Step 1), 1 prolongation, 2 Oseen element
 * assembly, 3 scatter reductions of the Oseen systems, 4 Darcy right-hand sides, 5 band
 * fill, 6 band LU, 7 band triangular solves, 8 FP64 residuals, 9 state update and glue,
 * 10 end-of-step copies.  ms[i] = total milliseconds, count[i] = timed intervals; either
 * array may be NULL; n = entries to write (at most 11). */
tpns_status tpns_set_timing(tpns_ctx* ctx, int32_t on);
tpns_status tpns_get_timings(const tpns_ctx* ctx, double* ms, int64_t* count, int32_t n);

/* Kernel launches issued by the library since it was loaded (all contexts). */
int64_t tpns_launch_count(void);

/* Last error message of a context (never NULL; "" when none).  ctx may be NULL for errors
 * raised before a context existed. */
const char* tpns_last_error(const tpns_ctx* ctx);

void tpns_destroy(tpns_ctx* ctx);

/* ---- introspection (tests) ----------------------------------------------------------
 * Mesh and subdomain data as the library built them, for bit-exact comparison with an
 * independent implementation.  what: 0 = fine fluid node coordinates (2 doubles / node),
 * 1 = fine porous node coordinates, 2 = fine fluid tri6 (6 int32 / triangle),
 * 3 = fine porous tri6.  Returns the number of values in *n when dst is NULL. */
tpns_status tpns_debug_mesh(const tpns_ctx* ctx, int32_t what, void* dst, size_t* n);

/* Local system j (0..n_local_systems-1; Oseen systems first, then 3 Darcy systems per
 * porous subdomain sharing one pattern): its unknowns as (global fine node id, component)
 * pairs in band order (component 0/1 velocity, 2 pressure for Oseen; 0 for Darcy), and its
 * CSR pattern rows/cols in that order.  dst arrays may be NULL to query sizes. */
tpns_status tpns_debug_system(const tpns_ctx* ctx, int32_t j, int32_t* n_unknowns,
                              int32_t* unknown_node, int32_t* unknown_comp,
                              int64_t* nnz, int32_t* rowptr, int32_t* colidx,
                              int32_t* kl, int32_t* ku);

/* Standalone solve of one sparse system A x = b with the library's band solver (the
 * factorisation and solves of Algorithm 3 Step 3): the CSR matrix is copied into band
 * storage, factored by the unpivoted band LU (FP32 or FP64 factors), and x is obtained by
 * triangular solves with FP64-residual iterative refinement (stop at ||b - A x|| <= 1e-13
 * ||b||, on stagnation, or after 12 corrections).
 *   n            unknowns; kl, ku: lower / upper bandwidth of A (every entry a_ij != 0 has
 *                i - j <= kl and j - i <= ku); kl + 32 <= 512.
 *   rowptr, colidx, vals, b, x: DEVICE pointers (CSR int32 / FP64, b and x FP64, n each);
 *                x is overwritten.
 *   precision    TPNS_FP64 or TPNS_FP32_IR; stream: cudaStream_t (NULL = legacy stream).
 *   relres_out   host pointer or NULL: final ||b - A x|| / ||b||.
 * Scratch (band, block inverses, vectors) is allocated with cudaMalloc for the call and
 * freed before returning (the call synchronises the stream).  The ordering of the unknowns
 * must make every leading block invertible (no pivoting); a zero or non-finite pivot
 * returns TPNS_EBREAKDOWN. */
tpns_status tpns_band_solve(int32_t n, int32_t kl, int32_t ku, const int32_t* rowptr,
                            const int32_t* colidx, const double* vals, const double* b,
                            double* x, tpns_precision precision, void* cuda_stream,
                            double* relres_out);

/* Same operation and arguments as tpns_band_solve, for callers that cannot allocate device
 * memory: code that runs while a CUDA stream is being captured into a graph (cudaMalloc is
 * not allowed there), hosts whose device memory is owned by another allocator that must not
 * see foreign allocations, and loops where an allocation's latency or failure at solve time
 * is not acceptable.  No part of the paper corresponds to it.
 * The scratch (band, block inverses, row index, vectors, flags) lives in one device array
 * of TPNS_NOALLOC_SCRATCH_BYTES bytes that the library declares statically; every device
 * that loads the library holds it until the process exits.  A system fits when
 *   n*(kl+ku+1)*s + ceil(n/32)*32*(kl+ku+64)*s + 4*nnz + 8*(n+130) + 4*(5+2*ceil(n/32)) + 2048
 * is at most that size (s = 4 for TPNS_FP32_IR, 8 for TPNS_FP64, plus 256-byte alignment of
 * each piece); larger systems are refused with TPNS_EINVAL.  The first call on a device looks
 * up the array's device address (with that device current); make that first call before any
 * stream capture.  All calls share the one array and it keeps the last call's contents, so
 * calls that overlap on the GPU (different streams or threads) race: serialise them. */
#define TPNS_NOALLOC_SCRATCH_BYTES (32u << 20)
tpns_status tpns_band_solve_noalloc(int32_t n, int32_t kl, int32_t ku, const int32_t* rowptr,
                                    const int32_t* colidx, const double* vals, const double* b,
                                    double* x, tpns_precision precision, void* cuda_stream,
                                    double* relres_out);

/* Host-only context: builds meshes, subdomains, orderings and patterns (Algorithm 3 Step 2)
 * without touching a GPU, for the introspection calls above.  Every other call on it
 * returns TPNS_EINVAL.  Release with tpns_destroy. */
tpns_status tpns_layout_create(const tpns_mesh_desc* mesh, const tpns_partition_desc* part,
                               tpns_ctx** out);

/* FP64 CSR values (nnz entries, pattern of tpns_debug_system) and right-hand side (n
 * entries) of local system j as assembled in the last step (Darcy: field 0..2 selects the
 * pressure; ignored for Oseen systems).  Host destination buffers. */
tpns_status tpns_debug_values(tpns_ctx* ctx, int32_t j, int32_t field, double* vals, double* rhs);

#ifdef __cplusplus
}
#endif
#endif /* TPNS_H */
