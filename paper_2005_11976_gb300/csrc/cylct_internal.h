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
};

// Volume tiling of the projector / back-projector: tt wedges x th slabs x all shells
// per tile (ragged last tiles), n_tt x n_th tiles, tile index = slab_tile * n_tt +
// wedge_tile.  One tile's voxels are staged in shared memory.
struct TileDev {
    int tt, th, n_tt, n_th, n_tiles;
    int smem_fp, smem_bp;   // dynamic shared memory bytes of the two kernels
};

// Device tables of one scan.
struct ScanDev {
    GridDev g;
    TileDev td;
    const float2 *trig;     // (cos, sin) of theta_k, k < N_theta
    const float4 *ray_a;    // ray records [view][pixel], see RayRec
    const float4 *ray_b;
    const float4 *ray_c;
    const int4 *bbox;       // candidate pixel box [view][tile]: u0, v0, u1, v1 (inclusive)
};

constexpr int kTileThreads = 256;

// SART update of one subset, fused into the back-projection epilogue.
struct UpdateArgs {
    float *x32;             // FP32 iterate (null in strict 16-bit mode)
    void *x16;              // 16-bit copy / iterate (null in FP32 mode)
    cyl_dtype x16_t;
    int strict16;
    const float *w;         // weight map or null
    const float *wscale;    // device scalar lambda / max(w) (or lambda), or null
    float lambda;
    int clamp;
};

// One scan of a batched solve (static for the whole solve).
struct BatchScan {
    ScanDev sd;
    const void *sino;       // [N_p][H][W] of the batch's sinogram dtype
    const void *x_proj;     // volume the projector reads (batch's projector dtype)
    UpdateArgs upd;         // fused update (16-bit dtype of the batch)
    float *q[2];            // two projection accumulators of subset_size x H x W
    int64_t q_len;
    float2 *nd[2];          // two (numerator, column sum) accumulators of N voxels
    int64_t nd_len;
};

// One unit of work of a round: subset [p0, p0 + np) of scan `scan`, accumulating into
// that scan's projection buffer q[buf].
struct BatchItem {
    int scan, p0, np, buf;
};

// Kernel launchers (kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_batch_round(const BatchScan *scans, const BatchItem *items, const int *n_items,
                               int max_items, int round, int max_tiles, int smem_fp, int smem_bp,
                               cyl_dtype xt, cyl_dtype st_, cyl_dtype x16t, cudaStream_t st);
cudaError_t launch_rays(const GridDev &g, const ProjGeom *geo, int n_proj, float4 *ra,
                        float4 *rb, float4 *rc, cudaStream_t st);
// q[v][pix] += sum over tiles of the tile's part of A x, views p0 .. p0+np-1 (q must be
// zeroed by the caller).
cudaError_t launch_fp_tiles(const ScanDev &sd, int p0, int np, const void *vol, cyl_dtype vt,
                            float *q, cudaStream_t st);
// SART mode (upd != null): residual (p - q) / L of the subset's rays back-projected into
// shared memory per tile, then the fused update of x.  Pure mode (upd == null): A^T y
// written to num_out and A^T 1 to den_out (if not null) for every voxel.
cudaError_t launch_bp_tiles(const ScanDev &sd, int p0, int np, const void *sino, cyl_dtype sdt,
                            const float *q, const UpdateArgs *upd, float *num_out,
                            float *den_out, cudaStream_t st);
cudaError_t launch_row_sums(const ScanDev &sd, int p0, int np, float *L, cudaStream_t st);
cudaError_t launch_count(const ScanDev &sd, int p0, int np, unsigned long long *counts,
                         cudaStream_t st);
cudaError_t set_kernel_attributes();

// Ray-piece kernels (rays.cu).  P = pieces per ray (1, 2, 4 or 8).
cudaError_t launch_fp_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt,
                           float *q, float2 *zero_buf, int64_t zero_len, cudaStream_t st);
// q != null: SART residual (y - q) / L into nd; q == null: pure A^T y into nd, or into
// num / den (den may be null) when nd is null.
cudaError_t launch_bp_rays(const ScanDev &sd, int P, int p0, int np, const void *y, cyl_dtype yt,
                           const float *q, float2 *nd, float *num, float *den, cudaStream_t st);
cudaError_t launch_update_nd(int64_t n_vox, const float2 *nd, const UpdateArgs &u, cudaStream_t st);
cudaError_t launch_count_rays(const ScanDev &sd, int p0, int np, unsigned long long *counts,
                              cudaStream_t st);
cudaError_t launch_batch_round_rays(const BatchScan *scans, const BatchItem *items, const int *n_items,
                                    int max_items, int round, int64_t max_rays, int64_t max_vox,
                                    int max_nt, int P, cyl_dtype xt, cyl_dtype yt, cyl_dtype x16t,
                                    cudaStream_t st);
cudaError_t launch_log(const void *in, cyl_dtype it, double i0, void *out, cyl_dtype ot,
                       int64_t n, cudaStream_t st);
cudaError_t launch_convert(const void *in, cyl_dtype it, void *out, cyl_dtype ot,
                           int64_t n, cudaStream_t st);
cudaError_t launch_weight_scale(const float *w, int64_t n, int mode, float lambda,
                                float *wscale, cudaStream_t st);

size_t dtype_size(cyl_dtype t);

}  // namespace cylct
