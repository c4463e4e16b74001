// Internal types shared by the CUDA translation units of libcylct.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/cylct.h"

namespace cylct {

// Per-projection ray geometry in the object frame (FP64): source S', centre D0' of
// pixel (0, 0), and the steps du', dv' from one pixel column / row to the next, so that
// pixel (iu, iv) sits at D0' + iu du' + iv dv'.
struct ProjGeom {
    double S[3];
    double D0[3];
    double du[3];
    double dv[3];
};

// Grid and detector constants for the kernels.
struct GridDev {
    int n_h, n_t, n_r;
    int det_w, det_h;
    int max_steps;          // bound on segments per ray (2 N_r + N_theta + N_h + 8)
    double radius, height;  // FP64 copies for the ray set-up
    double dr_d;            // FP64 shell spacing
    float dr, inv_dr;       // shell spacing
    float dth, inv_dth;     // wedge angle and its inverse
    float dh, inv_dh, h0;   // slab spacing, first slab plane (-H/2)
    float eps;              // floor of Eq. 7's row and column sums: 2^-16 radius
};

// Device tables of one scan.
struct ScanDev {
    GridDev g;
    const float2 *trig;     // (cos, sin) of theta_k, k < N_theta
    const float4 *ray_a;    // ray records [view][pixel], see RayRec
    const float4 *ray_b;
    const float4 *ray_c;
    const uint16_t *split;  // [view][pixel][kSplit]: cuts of each ray into kSplit pieces
                            // of equal step counts, as fractions of its chord / 65535
    int *sched;             // two self-resetting work counters per kernel kind (kSched)
};

// The rays of positive chord of a compact plan's pose, view by view in ray order (plan ray
// index); their records and cuts sit at their list positions.  act = null: a dense plan
// (every ray a task, records indexed by ray).  Passed to the ray kernels as their last
// argument.
struct RayList {
    const uint32_t *act;
    const int64_t *act_off;   // [n_proj + 1]: start of each view's rays in act
};

constexpr int kSplit = 16;  // pieces per ray recorded at set-up (P divides it)
constexpr int kPiecesFp = 8, kPiecesBp = 2;   // default pieces per ray of each kernel
constexpr int kSched = 10;  // ints of scheduler state per plan (two per ray kernel kind)
// The one-launch SART subset (k_sart): threads per block and default pieces per ray.
constexpr int kSartThreads = 128, kPiecesSart = 8;

// Stored segment records of a pose (records.cu): each ray's pieces as 4-byte records
// (FP32 length, low 3 bits the move to the next piece's voxel), cut into P runs of
// consecutive pieces; a task is 32 / P consecutive pixels of a view, one run per lane,
// whose records are rows of 32 words.
constexpr int kRecMoves = 8;
constexpr int kRecLgP = 3;    // default runs per ray: 8
struct RecDev {
    const uint32_t *rec;      // [rows][32]
    const int64_t *row_off;   // [n_tasks + 1]: first row of each task (task = view * tpv + pixel / R)
    const uint32_t *cnt;      // [view][pixel]: pieces of each ray
    const int32_t *idx0;      // [view][pixel][P]: voxel of the first piece of each run
    const float4 *ray_c;      // ray records' third part (chord = row sum L_j in .z)
    int64_t npix;
    int64_t tpv;              // tasks per view
    int lgP;                  // log2 of the runs per ray
    int delta[kRecMoves];     // voxel index change of each move code
    float eps;                // floor of Eq. 7's sums
};

// Transpose of a pose's records (gather.cu): per view and voxel, the (pixel, length) of
// every piece that crosses the voxel, for the back-projection by gathering per voxel.
struct VoxDev {
    const uint2 *ent;         // entries (pixel, FP32 length bits), view after view
    const int64_t *ebase;     // [n_proj + 1]: first entry of each view
    const uint32_t *off;      // [view][V + 1]: each voxel's first entry within its view
    int64_t n_vox, npix;
    float eps;                // floor of Eq. 7's sums
};

// SART update of one subset (Eq. 7): x += scale * w * num / den where den > 0.
struct UpdateArgs {
    float *x32;             // FP32 iterate (null in strict 16-bit mode)
    void *x16;              // 16-bit copy / iterate (null in FP32 mode)
    cyl_dtype x16_t;
    int strict16;
    const void *w;          // weight map (w_t elements) or null
    cyl_dtype w_t;
    const float *wscale;    // device scalar lambda / max(w) (or lambda), or null
    float lambda;
    int clamp;
    float den_eps;          // floor of the column sums (x += s w num / max(den, den_eps))
};

// One scan of a batched solve (static for the whole solve).
struct BatchScan {
    ScanDev sd;
    RayList rl;             // the scan's list of rays that meet its grid (act = null: dense)
    const void *sino;       // [N_p][H][W] of the batch's sinogram dtype
    const void *x_proj;     // volume the projector reads (batch's projector dtype)
    UpdateArgs upd;         // fused update (16-bit dtype of the batch)
    float *q[2];            // two projection accumulators of subset_size x H x W
    int64_t q_len;
    float2 *nd[2];          // two (numerator, column sum) accumulators of N voxels
    int64_t nd_len;
};

// One unit of work of a round: subset [p0, p0 + np) of scan `scan`, projecting into
// that scan's projection buffer q[buf] and back-projecting into nd[buf].
struct BatchItem {
    int scan, p0, np, buf;
};

// Kernel launchers.  All return cudaError_t of the launch.
// kernels.cu: ray records, row sums, elementwise kernels.
cudaError_t launch_rays(const GridDev &g, const ProjGeom *geo, int n_proj, float4 *ra,
                        float4 *rb, float4 *rc, cudaStream_t st);
cudaError_t launch_row_sums(const ScanDev &sd, int p0, int np, float *L, cudaStream_t st,
                            const RayList &rl = RayList{nullptr, nullptr});

// Ray-piece kernels (rays.cu).  P = pieces per ray: 1, 2, 4, 8 or 16 (a divisor of
// kSplit); P <= 0 means the kernel's default (kPiecesFp, kPiecesBp).
int valid_pieces(int P);
int default_pieces(int kind /* 0 forward, 1 back */);
// Cut every ray of all views into kSplit pieces of equal step counts (once per pose).
// cnt (if not null): each ray's number of pieces.
cudaError_t launch_split(const ScanDev &sd, int64_t n_rays, uint16_t *split, cudaStream_t st,
                         uint32_t *cnt = nullptr);   // n_rays records
// Compact plans: the rays of positive chord of every view, in ray order, with their
// records at their list positions.  Count (and scan into act_off), then fill.
constexpr int kActChunk = 1024;   // rays per block of the list's count and fill passes
cudaError_t launch_list_count(const GridDev &g, const ProjGeom *geo, int n_proj, int64_t *chunk, int64_t *act_off,
                              cudaStream_t st);
cudaError_t launch_list_fill(const GridDev &g, const ProjGeom *geo, int n_proj, const int64_t *chunk, int64_t cap,
                             uint32_t *act, float4 *ra, float4 *rb, float4 *rc, cudaStream_t st);
// Records of the n listed rays for a pose that differs from the list's pose by a spin only.
cudaError_t launch_list_refill(const GridDev &g, const ProjGeom *geo, const uint32_t *act, int64_t n, float4 *ra,
                               float4 *rb, float4 *rc, cudaStream_t st);
// q[v][pix] = (A x)_j for views p0 .. p0+np-1 (overwritten; in compact plans only the listed
// rays); zero_buf (if not null) is cleared on the way.
cudaError_t launch_fp_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt,
                           float *q, float2 *zero_buf, int64_t zero_len, cudaStream_t st,
                           const RayList &rl = RayList{nullptr, nullptr});
// q != null: SART residual (y - q) / L into nd; q == null: pure A^T y into nd, or into
// num / den (den may be null) when nd is null.  The outputs accumulate.
cudaError_t launch_bp_rays(const ScanDev &sd, int P, int p0, int np, const void *y, cyl_dtype yt,
                           const float *q, float2 *nd, float *num, float *den, cudaStream_t st,
                           const RayList &rl = RayList{nullptr, nullptr});
// One SART subset per launch (k_sart): the forward projection of views p0 .. p0+np-1,
// the residuals against y, and their back-projection into nd (the spare accumulator
// zero_buf cleared on the way).  P: pieces per ray (<= 0: kPiecesSart).
cudaError_t launch_sart_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt, const void *y,
                             cyl_dtype yt, float2 *nd, float2 *zero_buf, int64_t zero_len, cudaStream_t st,
                             const RayList &rl = RayList{nullptr, nullptr});
cudaError_t launch_update_nd(int64_t n_vox, const float2 *nd, const UpdateArgs &u, cudaStream_t st);
// Blocks of a persistent grid of `kernel`: every SM filled with as many blocks of
// `threads` threads (and `smem` bytes of dynamic shared memory) as fit, at most `cap`
// per SM (0: no cap); looked up once per kernel and device.
unsigned persistent_blocks(const void *kernel, size_t smem, int cap = 0, int threads = 256);
// Records (records.cu), 2^lgP runs per ray.  Count the pieces of every ray of views
// 0 .. n_proj-1 into cnt and the first row of each task into row_off (n_tasks + 1
// entries, row_off[n_tasks] = rows); then, with rec sized for those rows, write the
// records and the runs' first voxels (*bad set if a ray's pieces differ from its count).
cudaError_t launch_rec_count(const ScanDev &sd, int n_proj, int lgP, uint32_t *cnt, int64_t *row_off,
                             cudaStream_t st);
// The rows and row offsets from counts already in cnt (launch_rec_count without its walk).
cudaError_t launch_rec_rows(const ScanDev &sd, int n_proj, const uint32_t *cnt, int64_t *row_off, cudaStream_t st);
cudaError_t launch_rec_fill(const ScanDev &sd, int n_proj, int lgP, uint32_t *cnt, const int64_t *row_off,
                            uint32_t *rec, int32_t *idx0, int *bad, cudaStream_t st);
RecDev rec_dev(const ScanDev &sd, int lgP, const uint32_t *rec, const int64_t *row_off, const uint32_t *cnt,
               const int32_t *idx0);
// One SART subset of views p0 .. p0+np-1 from the records: the projections, the residuals
// against y and their back-projection into num (the numerator of Eq. 7, 4 ceil(V / 4)
// floats, 16-byte aligned); with resid (np x H x W floats) instead, the residuals are
// written there and nothing is back-projected.  sched: two ints of scheduler state, zero
// at rest.
cudaError_t launch_rec_sart(const RecDev &rd, int p0, int np, const void *x, cyl_dtype xt, const void *y,
                            cyl_dtype yt, float *num, float *resid, int *sched, cudaStream_t st);
// The reciprocal column sums r (4 ceil(V / 4) floats, 16-byte aligned) of the subset of
// views p0 .. p0+np-1 (Eq. 7's normalisation): each view's sums in FP32 into den32
// (4 ceil(V / 4) floats), added across the subset's views in FP64 into den64 (as many
// doubles; only used when np > 1).  Both must be zero on entry and are zero on return.
cudaError_t launch_rec_inv_den(const RecDev &rd, int p0, int np, int64_t n_vox, float *den32, double *den64,
                               float *r, cudaStream_t st);
// x += s w num r, num cleared.
cudaError_t launch_update_rec(int64_t n_vox, float *num, const float *r, const UpdateArgs &u, cudaStream_t st);
// Transpose (gather.cu), per pose: count the pieces of every voxel of every view and scan
// them into off ([view][V + 1]) and ebase ([n_proj + 1]; cnt: V, tsum: ceil(V / 2048)
// scratch); then, with ent sized for ebase[n_proj] entries (h_ebase: ebase on the host),
// fill the entries (cur: V scratch).
cudaError_t launch_vox_count(const RecDev &rd, int n_proj, int64_t n_vox, uint32_t *cnt, uint32_t *off,
                             uint32_t *tsum, int64_t *ebase, cudaStream_t st);
cudaError_t launch_vox_fill(const RecDev &rd, int n_proj, int64_t n_vox, const uint32_t *off, const int64_t *h_ebase,
                            uint32_t *cur, uint2 *ent, cudaStream_t st);
// Eq. 7 for the subset of views p0 .. p0+np-1 by gathering per voxel over the subset's
// residuals resid ([np][H][W]): back-projection, column sums and update in one pass.
cudaError_t launch_vox_sart(const VoxDev &vd, int p0, int np, const float *resid, const UpdateArgs &u,
                            cudaStream_t st);
cudaError_t launch_count_rays(const ScanDev &sd, int p0, int np, unsigned long long *counts,
                              cudaStream_t st,
                              const RayList &rl = RayList{nullptr, nullptr});
// One round of a batched solve: forward projection, back-projection and update of every
// item of the round (the kernels selected by `parts`; kRoundFused: projection, residual
// and back-projection in one launch with Pf pieces per ray).  Pf, Pb: pieces per ray of
// the two kernels (<= 0: their defaults).  sched: the batch's scheduler state (kSched
// ints, zero at rest).
constexpr int kRoundFp = 1, kRoundBp = 2, kRoundUpdate = 4, kRoundAll = 7, kRoundFused = 8;
cudaError_t launch_batch_round(const BatchScan *scans, const BatchItem *items, const int *n_items,
                               int max_items, int round, int64_t max_vox, int Pf, int Pb, int parts,
                               int *sched, cyl_dtype xt, cyl_dtype yt, cyl_dtype x16t, cudaStream_t st,
                               bool lists = false);
cudaError_t launch_log(const void *in, cyl_dtype it, double i0, void *out, cyl_dtype ot,
                       int64_t n, cudaStream_t st);
cudaError_t launch_convert(const void *in, cyl_dtype it, void *out, cyl_dtype ot,
                           int64_t n, cudaStream_t st);
cudaError_t launch_weight_scale(const void *w, cyl_dtype w_t, int64_t n, int mode, float lambda,
                                float *wscale, cudaStream_t st);

size_t dtype_size(cyl_dtype t);
// binaryVersion of the library's kernel image on the current device (e.g. 103)
cudaError_t kernel_binary_version(int *v);
// element types a weight map may have (sinograms and volumes: F32, F16, BF16 only)
inline bool valid_weight_dtype(int t) { return t == CYL_F32 || t == CYL_F16 || t == CYL_BF16 || t == CYL_U8; }

}  // namespace cylct
