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
 *     3D (tpns_mesh_desc.dim = 3): 0, 1, 2 = u_x, u_y, u_z, 3 = p, 4, 5, 6 = p_F, p_f, p_m;
 *     vertex (i, j, k) -> i + (nx+1) (j + (ny+1) k), then the edges of the Kuhn
 *     tetrahedra sorted by (min, max) vertex id.  Manufactured solutions: 1, 3 (2D), 2, 4
 *     (3D), 0 (zero data).
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
 * fine_rows_from_gamma[c] equal rows.
 * dim = 3 (Sec. 6 Example 2 geometry: porous box [0,1]^3 below the fluid box
 * [0,1]^2 x [1,2], Gamma at z = 1): uniform Kuhn tetrahedral meshes, coarse cells of edge
 * H = 1/nx_coarse (ny_coarse must equal nx_coarse), fine cells of edge H / fine_per_coarse_x;
 * fine_rows_from_gamma is not read.  dim = 0 or 2: the 2D meshes above. */
typedef struct {
  int32_t nx_coarse;
  int32_t ny_coarse;
  int32_t fine_per_coarse_x;
  int32_t fine_rows_from_gamma[TPNS_MAX_COARSE_ROWS];
  int32_t dim;
} tpns_mesh_desc;

/* Physical parameters of Sec. 2 (order of Darcy arrays: F, f, m). */
typedef struct {
  double nu, eta, rho, mu, alpha, sigma, sigma_star;
  double phiC[3];      /* phi_i C_i */
  double k[3];         /* permeabilities */
} tpns_params;

/* Algorithm 3 Step 2: nsub_x x nsub_y (x nsub_z in 3D) boxes D_j per region aligned with
 * coarse lines, enlarged by `overlap` fine layers on sides inside the region. */
typedef struct {
  int32_t nsub_x, nsub_y;
  int32_t overlap;
  int32_t nsub_z;      /* 3D only */
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
  double band_lu_flops;           /* algorithmic flops of one step's Oseen factorisations: band
                                     LU: sum over columns of l + 2 l u; multifrontal: sum over
                                     fronts and pivots of r + 2 r^2, r = rows below the pivot */
  int64_t h2d_bytes;              /* bytes copied host -> device by tpns_create */
  int64_t last_ir_solves;         /* band solve passes over all local systems, last step */
  double last_solve_bytes;        /* algorithmic bytes of those passes: per pass and system
                                     n (kl + ku) s + ceil(n / 32) 2048 s + 24 n, s = factor
                                     element size (factor slabs, diagonal-block inverses, FP64
                                     right-hand side read and solution read + write) */
  double last_step_ms;            /* device time of the context's last step in tpns_batch_step,
                                     from the step's start on its stream to its end (with the
                                     other contexts of the batch running beside it) */
  int64_t lu_cluster_ctas;        /* band LU: CTAs per cluster of the Oseen band LU, 8, or 16
                                     where all clusters fit the device and tpns_create measured
                                     16 faster on the context's own systems; 0 with the
                                     multifrontal factorisation */
  /* sizes of one step's local problems (for algorithmic byte counts) */
  int64_t oseen_unknowns, oseen_nnz, oseen_elements;   /* all local Oseen systems */
  int64_t darcy_unknowns, darcy_elements;             /* all local Darcy systems (x 3 fields) */
  double factor_entries;          /* stored entries of one step's Oseen factors (L and U) */
  int64_t mf_fronts;              /* multifrontal: fronts per step (0 with the band LU) */
  double create_ms;               /* host wall time of tpns_create for this context */
  int32_t last_gmres_outer;       /* GMRES-based refinement cycles run in the last step (0: none
                                     needed) */
  int32_t gmres_steps;            /* steps so far that needed them */
} tpns_stats;

typedef struct tpns_ctx tpns_ctx;

/* Factorisation of the local Oseen systems of Algorithm 3 Step 3(2) (eq. uclocalFully; the
 * paper leaves the solver open).  The Darcy systems always use the one-time band Cholesky. */
typedef enum {
  TPNS_FACTOR_MULTIFRONTAL = 0,   /* nested dissection of the subdomain's node grid, dense
                                     fronts factorised level by level (default) */
  TPNS_FACTOR_BAND = 1            /* unpivoted band LU in the band ordering */
} tpns_factor;

/* Options of tpns_create_ex; a zero-filled struct (or NULL) gives the defaults. */
typedef struct {
  int32_t local_factor;     /* tpns_factor */
  int32_t mf_leaf;          /* multifrontal: boxes of at most this many unknowns are not
                               dissected further (0 = 96) */
  int32_t mf_cuda_cores;    /* multifrontal, FP32 factors: 1 = trailing updates on the CUDA
                               cores; 0 = on the tensor cores (tcgen05, each operand split in
                               two TF32 parts, FP32 accumulation) */
  int32_t mf_ctas;          /* multifrontal: CTAs of the factorisation and solve launches
                               (0 = as many as are resident at once: one per SM for the
                               tensor-core factorisation) */
  int32_t rank, nranks;     /* split of one simulation over nranks contexts (one per GPU;
                               0 / 0 = whole simulation): the subdomains of each region are
                               assigned to ranks by estimated per-step work, largest first, each
                               to the least loaded rank (the same on every rank, no
                               communication); a context solves only its own subdomains and
                               replicates the coarse solve (Algorithm 3 Steps 1 and 3), and
                               tpns_get_field returns its part of the glued field: the sum over
                               ranks of the returned fields is the glued field of Step 4 (rank 0
                               adds the coarse interpolant).  nranks must not exceed the number
                               of subdomains per region. */
  int32_t algorithm;        /* 0 or 3: Algorithm 3 (two-grid, local parallel); 1: Algorithm 1
                               (Sec. 3.3: the decoupled partitioned time stepping on the fine
                               grid itself), run on the same kernels as Step 1 with the coarse
                               mesh set to the fine mesh (uniform fine rows only; the partition
                               is ignored; the whole fine problem must fit the coarse-solve
                               limits: Oseen system below about 25,000 unknowns in FP64) */
  int32_t refinement;       /* 0: classic iterative refinement x += (LU)^{-1} (b - A x), FP64
                               residuals, stop at the tolerance or on stagnation; 1: the same,
                               and when a local system is still above the tolerance after a
                               step's classic passes, restarted GMRES preconditioned by the
                               factors (FP64 Krylov vectors and Hessenberg problem; GMRES-based
                               refinement) corrects it before the corrections are glued; the
                               step then synchronises the stream to check */
  int32_t ir_classic_max;   /* classic refinement passes per step (0 = 12 for low-precision
                               factors, 2 for FP64) */
  int32_t mf_big_m;         /* multifrontal: fronts of at least this order, and all their
                               ancestors, are factored by all CTAs together, one height level
                               of the elimination trees at a time (0 = 256; < 0: never) */
} tpns_options;

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

/* tpns_create with options (see tpns_options; NULL = defaults).  TPNS_BF16_IR is available
 * with TPNS_FACTOR_BAND only. */
tpns_status tpns_create_ex(const tpns_mesh_desc* mesh, const tpns_params* params,
                           const tpns_partition_desc* part, const tpns_data_desc* data,
                           double dt, tpns_precision precision, size_t hbm_budget_bytes,
                           void* cuda_stream, const tpns_options* options, tpns_ctx** out);

/* Advance nsteps time steps (Algorithm 3 Steps 1, 3, 4 each step), enqueued on the
 * context's stream.  Cost on the host: after the last step is enqueued the call reads the
 * status words, refinement counters and residuals of every local system back (a few
 * device-to-host copies), so it synchronises the stream once per call; callers that want
 * work in flight across calls pass a larger nsteps. */
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

/* Number of global fine values of a field (see field ids above): the dimension of the
 * fine finite element space of that unknown (Sec. 3.2: X_h, Q_h for the conduit, X_ph for
 * each Darcy pressure), Dirichlet nodes included. */
tpns_status tpns_num_dofs(const tpns_ctx* ctx, int32_t field, size_t* n);

/* Copy the glued global fine field of the last step into dst (n values, FP64): the
 * corrected solution u^h = I_h u_H^{n+1} + sum_j w_j e_j^{n+1} of Algorithm 3 Step 4
 * ("correction of data"), in the global fine numbering.  n must equal tpns_num_dofs.
 * dst_on_device != 0: dst is a device pointer on the context's device (copied on the
 * context's stream, then the stream is synchronised); otherwise a host pointer. */
tpns_status tpns_get_field(tpns_ctx* ctx, int32_t field, double* dst, size_t n,
                           int32_t dst_on_device);

/* Counters of the last step and sizes of the context.  The paper has no counterpart: it
 * reports only run times (Sec. 6, Tables 1-4) and leaves the linear solvers unspecified;
 * these counters describe this library's factorisations and refinement. */
tpns_status tpns_get_stats(tpns_ctx* ctx, tpns_stats* out);

/* Serving: one time step of each of n contexts (Algorithm 3 Steps 1, 3, 4 of independent
 * simulations; the paper runs one simulation at a time, so batching them has no
 * counterpart there).  The steps of all contexts are enqueued
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
 * raised before a context existed or outside one; that message is kept per host thread.
 * No counterpart in the paper. */
const char* tpns_last_error(const tpns_ctx* ctx);

/* Release every device and host resource of a context (waits for its stream first).
 * NULL is ignored.  No counterpart in the paper. */
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
 *                i - j <= kl and j - i <= ku); kl + 32 <= 512 and ku + 32 <= 512.
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
 * memory: hosts whose device memory belongs to another allocator that must not see foreign
 * allocations, and loops where the latency or the failure of an allocation at solve time is
 * not acceptable.  No part of the paper corresponds to it.
 * The scratch (band, block inverses, solve vector, row index, vectors, flags) lives in one
 * device array of TPNS_NOALLOC_SCRATCH_BYTES bytes that the library declares statically;
 * every device that loads the library holds it until the process exits.  With s = 4 for
 * TPNS_FP32_IR and 8 for TPNS_FP64, a system fits when the sum of these pieces, each rounded
 * up to a multiple of 256 bytes,
 *   n*(kl+ku+1)*s  +  ceil(n/32)*2048*s  +  ceil(n/32)*32*kl*s  +  ceil(n/32)*32*ku*s
 *   + n*s  +  sizeof(SysDev) (< 256)  +  4*(6+2*ceil(n/32))  +  4*nnz  +  8*(n+130)
 * is at most that size; larger systems are refused with TPNS_EINVAL.  kl and ku are each at
 * most 480.  The call reads nnz from rowptr[n] and the final status back to the host and
 * synchronises the stream (also on every failure after its first launch), so when it
 * returns no work of it is still running.  The first call on a device looks up the array's
 * device address with that device current.  All calls share the one array and it keeps the
 * last call's contents, so calls that overlap on the GPU (issued from different host threads)
 * race: serialise them. */
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

/* tpns_layout_create with options (only local_factor and mf_leaf are read; NULL = defaults). */
tpns_status tpns_layout_create_ex(const tpns_mesh_desc* mesh, const tpns_partition_desc* part,
                                  const tpns_options* options, tpns_ctx** out);

/* Multifrontal structure of local Oseen system j (0 .. number of conduit subdomains - 1) as
 * the library analysed it, for an independent check of the symbolic factorisation.  what:
 *   0  [number of fronts, number of levels]
 *   1  per front (postorder, children before parents): m, p, level, parent, nchild,
 *      child0, child1 (7 int32; -1 = none)
 *   2  front rows: per front its m unknowns (system numbering of tpns_debug_system), own
 *      pivots first in elimination order, then the update set
 *   3  per front its update set mapped into the parent's rows (m - p int32)
 *   4  per front m + 1 column pointers into the front's originals (from 0)
 *   5  originals: CSR entry index within the system, per front and column
 *   6  originals: row of the entry in the front
 *   7  per front 2 m int32: column of child 0 / child 1 added into column j (or -1)
 *   8  elimination order (n unknowns)
 * Returns the number of int32 values in *n when dst is NULL.  TPNS_EINVAL without a
 * multifrontal analysis. */
tpns_status tpns_debug_fronts(const tpns_ctx* ctx, int32_t j, int32_t what, int32_t* dst, size_t* n);

/* FP64 CSR values (nnz entries, pattern of tpns_debug_system) and right-hand side (n
 * entries) of local system j as assembled in the last step (Darcy: field 0..2 selects the
 * pressure; ignored for Oseen systems).  Host destination buffers. */
tpns_status tpns_debug_values(tpns_ctx* ctx, int32_t j, int32_t field, double* vals, double* rhs);

#ifdef __cplusplus
}
#endif
#endif /* TPNS_H */
