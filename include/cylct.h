/*
 * cylct.h -- C ABI of the GB300 cylindrical-grid SART library (libcylct.so).
 *
 * Method: Goethals, Heyndrickx, Boone, "Fast tomographic inspection of cylindrical
 * objects" (J. Nondestructive Evaluation).  Cone-beam X-ray CT reconstructed by SART
 * (Eq. 7) on a cylindrical (N_h, N_theta, N_r) grid attached to the part's own axis
 * (Sec. 2, Eq. 1-2), with an initial volume and a weight map (Sec. 2.2, Sec. 3.3).
 *
 * Conventions (the paper leaves them open; every entry point uses these):
 *   - Lab frame: source at (-SOD, 0, 0); detector plane x = SDD - SOD, columns u along
 *     +y, rows v along +z; pixel (iu, iv) centre at
 *     (SDD - SOD, (iu - (W-1)/2) pitch_u + off_u, (iv - (H-1)/2) pitch_v + off_v).
 *   - Projection p: the stage is turned by angles_rad[p] about z; stage coordinates are
 *     X = Rz(-phi_p) X_lab.
 *   - Pose (Eq. 1): object coordinates X' = R (X - T), R the transpose of the intrinsic
 *     zxz orientation Rz(alpha) Rx(beta) Rz(gamma) (gamma spins the part about its own
 *     axis), T the part's position in stage coordinates, mm.
 *   - Grid (Eq. 2, theta = atan2(y', x') in [0, 2 pi)): shells r_k = k R / N_r, wedges
 *     theta_k = 2 pi k / N_theta, slabs h_k = -H/2 + k H / N_h.
 *   - Volumes are [N_h][N_theta][N_r] (r fastest), voxel l = (ih N_theta + it) N_r + ir.
 *     Sinograms are [N_p][H][W] (u fastest).  mu in 1/mm, lengths in mm.
 *   - System matrix (Sec. 2.2, Eq. 6): t_jl = exact length of ray j (source -> pixel
 *     centre) inside voxel l.
 *
 * Memory and ownership: the caller owns every array argument.  Unless an entry point
 * says otherwise, array pointers are DEVICE pointers on the plan's device.  The library
 * owns plans, their geometry tables and scratch, and servers.
 *
 * Streams: `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 * stream.  Calls are asynchronous on that stream unless stated otherwise.  A plan's
 * kernels run on the plan's own work stream, ordered after the work queued on `stream`
 * before the call and before the work queued on it after the call, so the calls of one
 * plan never overlap on the GPU whatever streams they are given.
 *
 * Errors: every int-returning call returns CYL_OK (0) or a negative CYL_E* code; no call
 * throws, prints, or aborts the process.  Arguments are validated on the host before any
 * work is queued.  cyl_last_error_detail() gives a one-line reason for the last failure
 * on the calling thread.
 */
#ifndef CYLCT_H
#define CYLCT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CYL_OK 0
#define CYL_EINVAL (-1)    /* invalid argument (sizes, geometry, pointers, dtype) */
#define CYL_ENOMEM (-2)    /* device or host allocation failed */
#define CYL_EDEVICE (-3)   /* a CUDA call failed */
#define CYL_EADMIT (-4)    /* request can never fit the server's HBM budget */
#define CYL_ETIMEOUT (-5)  /* a bounded wait ran out */
#define CYL_ENOTFOUND (-6) /* unknown ticket */
#define CYL_EPENDING (-7)  /* result not ready yet (cyl_poll) */
#define CYL_ECANCELLED (-8) /* request cancelled or server shut down */

/* Element types.  Sinograms and volumes: F32, F16 or BF16.  Weight maps (Sec. 2.2
 * weighted back-projection) also U8: a class map whose byte values are the weights. */
typedef enum { CYL_F32 = 0, CYL_F16 = 1, CYL_BF16 = 2, CYL_U8 = 3 } cyl_dtype;

/* Cylindrical grid about the part's axis (Sec. 2, Eq. 2). */
#define CYL_MAX_N_THETA 6144     /* the wedge (cos, sin) table is staged in 48 KB of shared memory */
typedef struct cyl_grid {
    int32_t n_h, n_theta, n_r;   /* slabs, wedges, shells; each >= 1; n_h <= 65535,
                                    n_theta <= CYL_MAX_N_THETA, n_r <= 65534 */
    double radius_mm, height_mm; /* grid cylinder: r <= radius, |h| <= height / 2 */
} cyl_grid;

/* Cone-beam acquisition.  Circular (Table 1 lists one such geometry): a fixed source and
 * detector and a turning stage, frames_mm = NULL.  General trajectory (a conveyor belt, a
 * helix): frames_mm holds, for each projection, 12 doubles in stage coordinates (no stage
 * turn): the source S, the centre D0 of pixel (0, 0) and the steps du, dv to the next
 * pixel column and row, mm; pixel (iu, iv) sits at D0 + iu du + iv dv.  With frames the
 * fields sod, sdd, pitch, off and angles are not used (angles_rad may be NULL).  Copied
 * at plan creation.  The server takes circular requests only. */
typedef struct cyl_geom {
    double sod_mm, sdd_mm;       /* 0 < sod < sdd */
    int32_t n_proj, det_w, det_h;
    double pitch_u_mm, pitch_v_mm, off_u_mm, off_v_mm;
    const double *angles_rad;    /* host array of n_proj stage angles; copied */
    const double *frames_mm;     /* NULL, or host array of n_proj x 12 (see above); copied */
} cyl_geom;

/* Part pose (Sec. 2, Eq. 1); see the conventions above. */
typedef struct cyl_pose {
    double alpha, beta, gamma;   /* radians */
    double tx, ty, tz;           /* mm */
} cyl_pose;

/* SART parameters (Eq. 7). */
typedef struct cyl_sart_params {
    int32_t n_iter;        /* full sweeps over all projections; >= 0 */
    int32_t subset_size;   /* consecutive projections per subset (OS); >= 1 */
    double lambda;         /* relaxation */
    int32_t clamp_nonneg;  /* 1: x = max(x, 0) after each update */
    int32_t weight_mode;   /* 1: w_hat = w / max(w); 0: w_hat = w */
    int32_t strict_16bit;  /* 16-bit x_out only: 1 = keep the iterate itself in 16 bits
                              (rounded after every subset); 0 = FP32 working iterate with a
                              16-bit copy that the projector reads */
    int32_t use_graph;     /* 1: replay each sweep as a captured CUDA graph */
    int32_t weight_dtype;  /* element type of the weight map: CYL_F32 (0), CYL_F16,
                              CYL_BF16 or CYL_U8; weights must be >= 0 */
} cyl_sart_params;

typedef struct cyl_plan cyl_plan;

/* One-line reason for the last failing call on this thread (static storage). */
const char *cyl_last_error_detail(void);
/* Name of a CYL_E* code. */
const char *cyl_strerror(int code);
/* Library version, e.g. "cylct 1.0". */
const char *cyl_version(void);

/* The compute capability the library's kernels were compiled for, as the runtime reports
 * it for `device` (major * 10 + minor: 103 for a GB300 build), in *binary_version.  Errors:
 * CYL_EINVAL (null output), CYL_EDEVICE (no such device, or the kernels have no image for
 * it).  A diagnostic: the paper has no counterpart. */
int cyl_binary_version(int device, int32_t *binary_version);

/* Create a plan for one scan: validates the grid, geometry and pose, builds the
 * per-projection ray tables (FP64, from the pose of Eq. 1, "only the alignment matrix
 * needs to be precomputed", Sec. 2.2) on `device` and allocates the scratch of a SART
 * solve.  *out receives the plan.  Errors: CYL_EINVAL, CYL_ENOMEM, CYL_EDEVICE. */
int cyl_plan_create(const cyl_grid *grid, const cyl_geom *geom, const cyl_pose *pose,
                    int device, cyl_plan **out);

/* Synchronises the plan's work and frees it.  NULL is accepted. */
int cyl_plan_destroy(cyl_plan *plan);

/* Re-pose a plan for the next scan of the same part type: rebuilds the per-projection
 * ray tables for `pose` (Eq. 1; the grid, geometry, scratch and any captured graph stay
 * resident, since the grid is fixed to the part, Sec. 2.2) and uploads them on `stream`,
 * ordered after the plan's earlier work.  Errors: CYL_EINVAL (non-finite pose),
 * CYL_EDEVICE. */
int cyl_plan_set_pose(cyl_plan *plan, const cyl_pose *pose, void *stream);

/* Eq. 6, left side: p = -ln(max(I, 1) / I0) for n detector values.  counts: array of
 * `in` type; p_out: array of `out` type; n >= 0.  Both are device memory or pinned
 * (page-locked) host memory, which the kernel reads or writes directly.  In-place
 * (counts == p_out, same dtype) is allowed. */
int cyl_log_transform(const void *counts, cyl_dtype in, double i0, void *p_out,
                      cyl_dtype out, int64_t n, void *stream);

/* Row sums L_j = sum_l t_jl (the denominator of Eq. 7's row normalisation) of the rays
 * of projections p0 .. p0+np-1, as the FP64 chord of each ray through the grid cylinder
 * rounded to FP32.  L_out: device float[np][H][W]. */
int cyl_row_sums(cyl_plan *plan, int32_t p0, int32_t np, float *L_out, void *stream);

/* Forward projection q = A x (Eq. 6 right side) for projections p0 .. p0+np-1.
 * vol: device [N_h][N_theta][N_r] of vol_dtype.  sino_out: device [np][H][W] of
 * sino_dtype (FP32 accumulation, rounded once on store). */
int cyl_project(cyl_plan *plan, const void *vol, cyl_dtype vol_dtype, int32_t p0,
                int32_t np, void *sino_out, cyl_dtype sino_dtype, void *stream);

/* Allocation-free forward projection.  The paper has no counterpart: this entry point
 * serves callers that must not allocate device memory while they run, such as a host
 * framework that owns all device memory through its own caching allocator, or an in-line
 * inspection loop that cannot afford an allocation (and the synchronisation it may bring)
 * between two parts.  Same arguments and result as cyl_project, but the FP32 accumulator
 * is a fixed array in the library's static device memory (CYL_NOALLOC_MAX_ELEMS floats,
 * 16 MiB, held on every GPU that loads the library until the process exits), so the call
 * makes no allocation at all.  np * H * W above CYL_NOALLOC_MAX_ELEMS gives CYL_EINVAL.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every call
 * shares the one array (each call overwrites it): calls of different plans that overlap
 * on the GPU, from any stream or thread, race and corrupt each other's results (calls of
 * one plan run in order on the plan's own work stream). */
#define CYL_NOALLOC_MAX_ELEMS (4 * 1024 * 1024)
int cyl_project_noalloc(cyl_plan *plan, const void *vol, cyl_dtype vol_dtype, int32_t p0,
                        int32_t np, void *sino_out, cyl_dtype sino_dtype, void *stream);

/* Matched back-projection out = A^T y over projections p0 .. p0+np-1 (the transpose of
 * exactly the t_jl cyl_project uses; Sec. 2.2 back-projection).  sino: device [np][H][W]
 * of sino_dtype.  vol_out: device float volume, OVERWRITTEN with A^T y.  colsum_out:
 * NULL or device float volume, overwritten with A^T 1 (Eq. 7's column sums). */
int cyl_backproject(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, int32_t p0,
                    int32_t np, float *vol_out, float *colsum_out, void *stream);

/* SART (Eq. 7) over all projections: x0 (warm start, Sec. 2.2 / 3.3 "initial volume";
 * NULL = zeros), weight map w (weighted back-projection, Sec. 2.2; NULL = none; of
 * params->weight_dtype),
 * n_iter sweeps of ordered subsets in index order; the result goes to x_out.
 *   sino:  [N_p][H][W] line integrals of sino_dtype;
 *   x0:    [N_h][N_theta][N_r] of x_dtype, or NULL;
 *   w:     [N_h][N_theta][N_r] of params->weight_dtype (>= 0), or NULL;
 *   x_out: [N_h][N_theta][N_r] of x_dtype (may equal x0).
 * Pointers may be device or host memory (each is checked); host arrays are staged
 * through plan-owned device buffers and the call then returns after x_out is written.
 * Rays with L_j = 0 contribute nothing; voxels no ray of a subset touches keep their
 * value.  Errors: CYL_EINVAL, CYL_ENOMEM, CYL_EDEVICE. */
int cyl_sart_solve(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, const void *x0,
                   const void *w, const cyl_sart_params *params, void *x_out,
                   cyl_dtype x_dtype, void *stream);

/* Batched SART: n scans (0 <= n <= CYL_MAX_BATCH; each its own plan: own pose,
 * projection count and geometry, all on one device) reconstructed together, each exactly
 * as cyl_sart_solve would with the same params.  A round advances every unfinished scan
 * by one subset: one forward projection and one back-projection launch take the ray
 * pieces of all the round's scans from a shared work counter, then the Eq. 7 update runs
 * per scan; all rounds are queued as one CUDA graph (params->use_graph).  The plans'
 * piece settings are those of plans[0].
 * Arrays (per scan i, in plan i's layout): sinos[i] of sino_dtype, x0s[i] (x0s or its
 * entries NULL = zeros), ws[i] weights of params->weight_dtype (ws or its entries NULL =
 * none), x_outs[i] of
 * x_dtype.  All DEVICE pointers on the plans' device; host arrays give CYL_EINVAL.
 * Asynchronous on `stream`.  Errors: CYL_EINVAL, CYL_ENOMEM, CYL_EDEVICE. */
#define CYL_MAX_BATCH 4096
int cyl_sart_solve_batch(int32_t n, cyl_plan *const *plans, const void *const *sinos,
                         cyl_dtype sino_dtype, const void *const *x0s, const void *const *ws,
                         const cyl_sart_params *params, void *const *x_outs, cyl_dtype x_dtype,
                         void *stream);

/* Autotuner of a batch: takes the arguments of cyl_sart_solve_batch, builds the same
 * rounds and times the first round's projector and back-projector for 1, 2, 4, 8 and 16
 * pieces per ray; the fastest setting of each is stored in plans[0] (which the batch
 * uses; cyl_plan_get_pieces reports it).  Writes only the plans' scratch (the outputs
 * and the iterate are not touched).  Synchronises the plans' work.  Errors as for
 * cyl_sart_solve_batch. */
int cyl_sart_tune_batch(int32_t n, cyl_plan *const *plans, const void *const *sinos,
                        cyl_dtype sino_dtype, const void *const *x0s, const void *const *ws,
                        const cyl_sart_params *params, void *const *x_outs, cyl_dtype x_dtype,
                        void *stream);

/* ---------------------------------------------------------------- serving
 * A server reconstructs a stream of in-line inspection scans of registered part types
 * (Sec. 2.4 / 3.3: series of same-type parts, each with its own pose; the grid is fixed to
 * the part, so one warm-start volume and one weight map per part type stay resident).
 * A scheduler thread runs continuous batching: each round advances every active scan by
 * one SART subset with the batched kernels, and requests that arrive while others are on
 * the GPU join at the next round as soon as their device footprint fits the HBM budget.
 * Every scan gets exactly the arithmetic of cyl_sart_solve with the server's parameters.
 */
typedef struct cyl_server cyl_server;

typedef struct cyl_server_cfg {
    int32_t device;
    int64_t hbm_budget_bytes;   /* device bytes the server may hold (parts + scans), > 0 */
    int32_t max_active;         /* scans reconstructed together, 1 .. 1024 */
    int32_t n_iter;             /* SART sweeps per scan */
    int32_t subset_size;
    double lambda;
    int32_t weight_mode;
    int32_t clamp_nonneg;
    cyl_dtype storage;          /* dtype of sinograms and volumes (F32, F16 or BF16) */
    int32_t rounds_ahead;       /* rounds queued on the GPU before the scheduler waits,
                                   1 .. 64 (0 = 4) */
    int32_t weight_dtype;       /* element type of the parts' weight maps (as in
                                   cyl_sart_params; 0 = CYL_F32) */
} cyl_server_cfg;

/* A request: one scan of a registered part type.  sino ([n_proj][H][W] line integrals of
 * the server's storage dtype) and x_out ([N_h][N_theta][N_r] of the storage dtype) may be
 * host or device memory; both must stay valid until cyl_poll reports completion.
 * angles_rad (n_proj stage angles) is copied by cyl_submit. */
typedef struct cyl_request {
    int32_t part;
    cyl_pose pose;
    int32_t n_proj;
    const double *angles_rad;
    const void *sino;
    void *x_out;
} cyl_request;

typedef struct cyl_result {
    int32_t status;             /* CYL_OK, CYL_EPENDING, or the error the scan ended with */
    int64_t submit_ns;          /* steady-clock times: submitted, admitted, result written */
    int64_t admit_ns;
    int64_t done_ns;
} cyl_result;

typedef struct cyl_server_stats {
    int64_t submitted, completed, failed, active, queued;
    int64_t rounds;             /* GPU rounds launched */
    int64_t hbm_in_use;         /* bytes held by parts and admitted scans */
} cyl_server_stats;

/* Start a server and its scheduler thread.  Errors: CYL_EINVAL, CYL_EDEVICE, CYL_ENOMEM. */
int cyl_server_create(const cyl_server_cfg *cfg, cyl_server **out);

/* Register a part type: its grid, its acquisition geometry (geom->n_proj and
 * geom->angles_rad are ignored: every request brings its own), a warm-start volume x0
 * (storage dtype, NULL = zeros) and a weight map w (cfg->weight_dtype, NULL = none), host or device
 * memory, copied into resident device memory.  *part receives the part id.  Errors:
 * CYL_EINVAL, CYL_EADMIT (the part alone exceeds the budget), CYL_ENOMEM, CYL_EDEVICE. */
int cyl_server_add_part(cyl_server *srv, const cyl_grid *grid, const cyl_geom *geom,
                        const void *x0, const void *w, int32_t *part);

/* Queue a request; *ticket identifies it.  Never blocks on the GPU.  Errors: CYL_EINVAL,
 * CYL_EADMIT (the scan can never fit the budget next to the resident parts),
 * CYL_ECANCELLED (server shutting down). */
int cyl_submit(cyl_server *srv, const cyl_request *req, uint64_t *ticket);

/* Result of a ticket: CYL_OK once done (out filled, the ticket is then released),
 * CYL_EPENDING while queued or running, CYL_ENOTFOUND for unknown or released tickets,
 * or the scan's error. */
int cyl_poll(cyl_server *srv, uint64_t ticket, cyl_result *out);

/* Like cyl_poll, but waits up to timeout_ms for completion; CYL_ETIMEOUT if it is still
 * pending then. */
int cyl_wait(cyl_server *srv, uint64_t ticket, int64_t timeout_ms, cyl_result *out);

int cyl_server_get_stats(cyl_server *srv, cyl_server_stats *out);

/* Stop the scheduler (queued requests end with CYL_ECANCELLED, running ones finish),
 * release all device memory and free the server.  NULL is accepted. */
int cyl_server_destroy(cyl_server *srv);

/* Segments (pieces of positive length between consecutive crossings, i.e. the
 * non-zero entries of each row of A counted with multiplicity) of each projection
 * p0 .. p0+np-1.  counts_out: device int64[np].  Used to state algorithmic bytes. */
int cyl_count_segments(cyl_plan *plan, int32_t p0, int32_t np, int64_t *counts_out,
                       void *stream);

/* Per-kernel device time of the plan's last cyl_sart_solve run with timing enabled.
 * kind: 0 forward projection, 1 back-projection, 2 update.  Timing records a CUDA event
 * between every two launches of a sweep.  With params->use_graph (and one captured
 * graph: an even number of subsets, or one sweep) the events are captured into the
 * sweep's graph and the times are those of the solve's last sweep; otherwise the
 * launches are eager and the times cover every sweep.  ms_total and launches receive
 * the sum of event durations and the number of launches timed. */
int cyl_plan_set_timing(cyl_plan *plan, int enable);
int cyl_plan_kernel_time(cyl_plan *plan, int kind, double *ms_total, int64_t *launches);

/* Work split of the projector and the back-projector: at set-up (plan creation and
 * cyl_plan_set_pose) each ray is walked once and cut into 16 pieces holding equal numbers
 * of steps; a launch runs P pieces per ray (P in 1, 2, 4, 8, 16; each piece one thread),
 * merging adjacent pieces for P < 16; the P pieces of a ray run in adjacent lanes of
 * one warp.  Defaults: 8 for the projector, 2 for the back-projector.
 * cyl_plan_tune times one view (view 0) with each P and keeps the fastest for this plan,
 * for the projector, the back-projector and the one-launch subset (cyl_plan_set_fused);
 * synchronises `stream`.  cyl_plan_set_pieces fixes P (0 restores the default);
 * cyl_plan_get_pieces reports the P in use. */
int cyl_plan_tune(cyl_plan *plan, void *stream);
/* How cyl_sart_solve runs a subset of Eq. 7.  enable = 1 (the default): one launch per
 * subset; the lanes of each ray walk it forward for its projection (Eq. 6), form its
 * residual, and walk it again to back-project the residual (kind 0 of
 * cyl_plan_kernel_time; kind 1 then has no launches).  enable = 0: a projector launch and
 * a back-projector launch (kinds 0 and 1), with the projections stored in between.  Both
 * give the same iterates to rounding.  Errors: CYL_EINVAL (null plan). */
int cyl_plan_set_fused(cyl_plan *plan, int32_t enable);
/* Pieces per ray of the one-launch subset (P as for cyl_plan_set_pieces; 0 restores the
 * default, 8).  Errors: CYL_EINVAL (null plan, P not 0 or a power of two up to 16). */
int cyl_plan_set_sart_pieces(cyl_plan *plan, int32_t pieces);
/* Stored segment records (Eq. 6: each ray's row of the system matrix, t_jl and voxel l of
 * every piece).  Every subset of Eq. 7 needs each of its rays' rows twice, for q_j and
 * for the back-projection of r_j, and the rows depend only on the pose.  enable = 1 or
 * 2: at this call and at every later cyl_plan_set_pose, each ray is walked once and its
 * pieces are written as 4-byte records (the FP32 length rounded to 20 mantissa bits,
 * relative error <= 2^-21, with the move to the next piece's voxel in the low 3 bits);
 * the one-launch subsets of cyl_sart_solve then replay the records instead of walking
 * each ray twice.
 *   enable = 1: the records are also transposed (per view and voxel, the pixel and
 *     length of every piece that crosses the voxel), and a subset is the records'
 *     forward replay for the residuals, then one pass over the voxels that gathers the
 *     back-projection and the column sums of Eq. 7 and updates x, without atomics.
 *     Where the transpose does not fit, as for enable = 2.
 *   enable = 2: the back-projection replays the records again into a numerator, with
 *     the column sums summed once per pose and subset size.
 * runs (0: the default, 8; else 1, 2, 4, 8, 16 or 32) cuts each ray's pieces into that
 * many runs of consecutive pieces, replayed side by side by as many warps.  The records
 * take about 4 bytes per piece of the whole scan (about 16 GB for 180 views of a
 * 256 x 256 detector through a (128, 512, 128) grid), the transpose about 8 bytes per
 * piece and 4 per voxel and view (about 33 GB there), the column sums of enable = 2 4
 * bytes per voxel and subset; the records are kept only where they fit within 40 % of
 * the device, the transpose where records and transpose fit within half of it, each
 * with 1 GiB free beside them, and otherwise the subsets walk the rays
 * (cyl_plan_records reports which).  Dense plans only (compact plans walk); the
 * two-launch form (cyl_plan_set_fused(0)), the projector and the back-projector always
 * walk.  enable = 0 (the default) frees them.  Synchronises `stream`.  Errors:
 * CYL_EINVAL (null plan, enable not 0, 1 or 2, runs not as above), CYL_EDEVICE. */
int cyl_plan_set_records(cyl_plan *plan, int32_t enable, int32_t runs, void *stream);
/* ready = 1 if the plan holds the records of its current pose, rec_bytes their size;
 * gather = 1 if it also holds their transpose (the gather form), gather_bytes its size.
 * Any output may be null. */
int cyl_plan_records(const cyl_plan *plan, int32_t *ready, int64_t *rec_bytes, int32_t *gather,
                     int64_t *gather_bytes);
int cyl_plan_set_pieces(cyl_plan *plan, int32_t fp_pieces, int32_t bp_pieces);
int cyl_plan_get_pieces(const cyl_plan *plan, int32_t *fp_pieces, int32_t *bp_pieces);

/* Sizes of a plan: voxels, rays per projection, projections, and the device bytes the
 * plan holds. */
int cyl_plan_sizes(const cyl_plan *plan, int64_t *n_vox, int64_t *n_pix, int32_t *n_proj,
                   int64_t *device_bytes);

/* ------------------------------------------------------------------------------------
 * Pose estimation from the projections (Sec. 2.1, "Projection based pose estimation").
 *
 * These calls need no plan and no grid: they take the acquisition geometry alone and run
 * on the calling thread's current CUDA device, where the sinograms must live.  Stage
 * coordinates are those of the conventions above (X = Rz(-phi_p) X_lab; with frames_mm,
 * the frames' own coordinates).
 *
 * Axis tracking.  In every projection the segment is the set of pixels with p > threshold
 * inside a detector window, dilated with the (2k+1) x (2k+1) square (clipped to the
 * window).  The test is exact: the stored value (FP32, FP16 or BF16) against the double
 * threshold, as if both were FP64 (the kernel compares in FP32 against the largest float
 * at or below the threshold, which decides every float alike).  Its four corner pixels are the extremes along the detector diagonals:
 * top-left maximises -iu + iv, top-right iu + iv, bottom-left -iu - iv, bottom-right
 * iu - iv (ties go to the larger iv for the top corners and the smaller iv for the
 * bottom ones).  The centre of the two top corners and the centre of the two bottom
 * corners lie on the projected symmetry axis; over the projections they form two tracks.
 *
 * Point tracking (Eq. 3-4).  Each track's 3-D point is the stage point X minimising
 * sum_i |(u, v)_i - V_i(X)|^2, with V_i(X) the detector position (mm along the pixel
 * steps) where the line from projection i's source through X meets the detector.
 * Levenberg-Marquardt with the analytic Jacobian of V_i, in FP64: start on the first
 * tracked projection's ray at the stage origin's distance from its source; damping mu =
 * 1e-3 on the diagonal of J^T J, divided by 10 after an accepted step (not below 1e-15)
 * and multiplied by 10 after a rejected one; stop after a step (accepted or not) shorter
 * than 1e-10 (1 + |X|) mm, when mu exceeds 1e15, or after max_iter steps.
 *
 * Pose.  The two axis points fix five of the six degrees of freedom of Eq. 1: the axis
 * direction a = (top - bottom) / |top - bottom| = (sin alpha sin beta,
 * -cos alpha sin beta, cos beta) gives alpha and beta (alpha = 0 when the axis is
 * vertical), the midpoint of the points gives T.  gamma, the spin about the part's own
 * axis, does not show in a silhouette; it is copied from the parameters (see
 * cyl_estimate_gamma).
 * ------------------------------------------------------------------------------------ */
#define CYL_MAX_DET_SIDE 262143      /* det_w, det_h limit of the corner keys (2^18 - 1) */
typedef struct cyl_pose_params {
    double threshold;     /* segment: p > threshold, in the sinogram's units */
    int32_t dilate_px;    /* k: 0 .. 65535 */
    int32_t roi[4];       /* window [u0, u1) x [v0, v1) in pixels; all 0 = whole detector */
    int32_t max_iter;     /* Levenberg-Marquardt steps per point; <= 0 selects 100 */
    double gamma;         /* copied into the estimated pose */
} cyl_pose_params;

typedef struct cyl_pose_info {
    double top_mm[3], bottom_mm[3];  /* tracked axis points, stage coordinates */
    double rms_mm[2];                /* rms detector distance between each track and V_i */
    int32_t iters[2];                /* Levenberg-Marquardt steps taken per point */
    int32_t n_views;                 /* projections whose window held a segment */
    int32_t status;                  /* 0: estimated; 1: fewer than 2 such projections (the
                                        pose is then the input gamma and zeros) */
} cyl_pose_info;

/* Corner pixels of every projection.  sino: device [n_proj][H][W] of sino_dtype.
 * corners_out: device int32[n_proj][4][2], (iu, iv) of the top-left, top-right,
 * bottom-left and bottom-right corners, (-1, -1) where the window holds no segment.
 * counts_out: device int64[n_proj] (pixels over the threshold, before dilation), or NULL.
 * Asynchronous on `stream`.  Errors: CYL_EINVAL (geometry, window, parameters, det_w or
 * det_h above CYL_MAX_DET_SIDE), CYL_ENOMEM, CYL_EDEVICE. */
int cyl_axis_corners(const cyl_geom *geom, const void *sino, cyl_dtype sino_dtype,
                     const cyl_pose_params *params, int32_t *corners_out, int64_t *counts_out,
                     void *stream);

/* Eq. 4 for one track.  track: device double[n_proj][2], the pixel coordinates (iu, iv)
 * of the point in each projection; NaN in either marks a projection where it was not
 * seen.  out: device double[5] = x, y, z (stage, mm), rms distance (mm), steps taken;
 * with fewer than 2 observed projections out is x = y = z = rms = NaN, steps = 0.
 * Asynchronous on `stream`. */
int cyl_track_point(const cyl_geom *geom, const double *track, int32_t max_iter, double *out,
                    void *stream);

/* The whole estimate for one scan: corners, both tracks, Eq. 4 for each, and the pose.
 * pose_out and info_out (may be NULL) are HOST structs; the call synchronises `stream`. */
int cyl_estimate_pose(const cyl_geom *geom, const void *sino, cyl_dtype sino_dtype,
                      const cyl_pose_params *params, cyl_pose *pose_out, cyl_pose_info *info_out,
                      void *stream);

/* n scans in one pass (one corner launch over all projections of all scans, one
 * Levenberg-Marquardt launch).  geoms, sinos, params: host arrays of n; poses_out,
 * infos_out (may be NULL): host arrays of n.  0 <= n <= CYL_MAX_BATCH.  Synchronises
 * `stream`. */
int cyl_estimate_pose_batch(int32_t n, const cyl_geom *geoms, const void *const *sinos,
                            cyl_dtype sino_dtype, const cyl_pose_params *params,
                            cyl_pose *poses_out, cyl_pose_info *infos_out, void *stream);

/* Device time of the pose kernels in the calls that synchronise (cyl_estimate_pose,
 * cyl_estimate_pose_batch): kind 0 the corner pass, 1 the Levenberg-Marquardt pass.  A
 * CUDA event pair on the call's stream brackets each launch while timing is enabled
 * (process-wide); cyl_pose_set_timing also resets the totals.  ms_total and launches
 * receive the summed durations and the number of launches timed. */
int cyl_pose_set_timing(int enable);
int cyl_pose_kernel_time(int kind, double *ms_total, int64_t *launches);

/* ------------------------------------------------------------------------------------
 * Azimuthal phase (Sec. 2.1, "Azimuthal phase", Eq. 5).
 *
 * The grey values of a band along the projected axis are followed over the projection
 * angle.  The band holds the pixels whose position, measured from the projection A of
 * the axis point (0, 0, h_lo) towards the projection B of (0, 0, h_hi), lies between A and
 * B (0 <= s <= 1) and within half_width of the line AB (|d| <= half_width, d in mm on the
 * detector, positive towards +u).  Per projection the library forms the band's grey-value
 * sum m0 = sum p and first moment m1 = sum p d, and the centroid offset c = m1 / m0.
 * Material off the axis pulls c to its side in a sine of the projection angle; the
 * first-harmonic phase phi_P of c (least-squares fit c ~ c0 + c1 cos phi + c2 sin phi,
 * phi_P = atan2(c2, c1)) moves with the part's spin gamma.
 *
 * s and d are evaluated in FP32 with rounding to nearest and no contraction:
 * d = (iu - A_u) c_du + (iv - A_v) c_dv, s = (iu - A_u) c_su + (iv - A_v) c_sv, with FP32
 * constants rounded from FP64 (c_du = |du| L_v / |L|, c_dv = -|dv| L_u / |L|,
 * c_su = |du| L_u / |L|^2, c_sv = |dv| L_v / |L|^2, L = B - A in mm).
 * ------------------------------------------------------------------------------------ */
typedef struct cyl_band {
    double h_lo_mm, h_hi_mm;   /* axis segment in object heights, h_lo < h_hi */
    double half_width_mm;      /* > 0 */
} cyl_band;

/* Band moments of a sinogram for a posed part.  moments_out: device double[n_proj][2] =
 * (m0, m1).  Asynchronous on `stream`. */
int cyl_band_moments(const cyl_geom *geom, const cyl_pose *pose, const void *sino,
                     cyl_dtype sino_dtype, const cyl_band *band, double *moments_out,
                     void *stream);

/* Eq. 5 with the tilt correction applied exactly.  The centroid moves furthest to +u for
 * material at lab azimuth phi_G = 90 deg, so material at stage azimuth psi peaks at
 * phi_P = phi_G - psi (stage turning counter-clockwise, as in the conventions above).
 * The stage azimuth psi of a direction at angle e from the line of nodes in the part's
 * tilted plane is psi = alpha + atan2(cos beta sin e, cos e), so
 * e(phi_P) = atan2(sin(phi_G - phi_P - alpha), cos beta cos(phi_G - phi_P - alpha)).
 * With phi_P_ref the phase of a reference whose spin is gamma_ref,
 * gamma = gamma_ref + e(phi_P) - e(phi_P_ref), wrapped to (-pi, pi].  (Eq. 5 as printed,
 * gamma = phi_P - phi_G - arctan(tan alpha / cos beta), is this relation with the phase
 * read in the tilted plane from the direction above the stage x axis and the stage
 * turning the other way.)  Host-only arithmetic. */
int cyl_gamma_from_phase(double phi_p, double phi_p_ref, double alpha, double beta,
                         double gamma_ref, double *gamma_out);

/* Spin of the scanned part relative to a template (the initial volume of Sec. 2.2).  The
 * plan must be posed with the part's alpha, beta and T (from cyl_estimate_pose) and a
 * starting reference spin as gamma; its geometry must be circular.  The call projects,
 * at the plan's pose, the template and its azimuthal mean (the axisymmetric part, whose
 * centroid signal holds the geometric terms of an off-centre part); takes the phases of
 * (c_scan - c_mean) and (c_template - c_mean); and converts them by cyl_gamma_from_phase.
 * Each further pass (passes > 1) re-poses the template at the current estimate and
 * repeats: on a partial arc (Table 1: 200 deg) the first-harmonic fits of two signals of
 * different phase pick up different shares of their higher harmonics, and the bias
 * vanishes as the reference's phase approaches the scan's.  On return the plan is posed
 * with the estimated gamma (no change for passes = 1 when the estimate equals the
 * starting spin).  sino: device [n_proj][H][W] of sino_dtype; tmpl: device volume of
 * tmpl_dtype; passes: 1 .. 16.  gamma_out: HOST double, the part's gamma.  diag_out: HOST
 * double[4] = phi_P, amplitude, phi_P_ref, reference amplitude of the last pass
 * (amplitudes in mm), or NULL.  Uses the plan's scratch; synchronises `stream`.  Errors:
 * CYL_EINVAL (frames geometry, band, passes), CYL_ENOMEM, CYL_EDEVICE. */
int cyl_estimate_gamma(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, const void *tmpl,
                       cyl_dtype tmpl_dtype, const cyl_band *band, int32_t passes, double *gamma_out,
                       double *diag_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
