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
    float inv_dth;          // 1 / wedge angle
    float dh, inv_dh, h0;   // slab spacing, first slab plane (-H/2)
};

// Ray-tile shape of the ray-driven kernels: a warp covers wu x (32 / wu) pixels, a
// block stacks 4 warps along v.
struct TileShape {
    int wu;
};

inline dim3 ray_block() { return dim3(128, 1, 1); }

// One subset of a SART sweep or one batched step: which projections, and where.
struct SubsetArgs {
    int p0, np;
};

// Kernel launchers (kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_project(const GridDev &g, const ProjGeom *geo, const float2 *trig,
                           int p0, int np, const void *vol, cyl_dtype vt, void *out,
                           cyl_dtype ot, TileShape ts, cudaStream_t st);
cudaError_t launch_residual(const GridDev &g, const ProjGeom *geo, const float2 *trig,
                            int p0, int np, const void *vol, cyl_dtype vt,
                            const void *sino, cyl_dtype sdt, int64_t sino_proj_stride,
                            float *res, TileShape ts, cudaStream_t st);
cudaError_t launch_backproject(const GridDev &g, const ProjGeom *geo, const float2 *trig,
                               int p0, int np, const void *y, cyl_dtype yt, float *num,
                               float *den, TileShape ts, cudaStream_t st);
cudaError_t launch_update(int64_t n_vox, float *x32, void *x16, cyl_dtype x16t,
                          int strict16, float *num, float *den, const float *w,
                          const float *wscale, float lambda, int clamp, cudaStream_t st);
cudaError_t launch_row_sums(const GridDev &g, const ProjGeom *geo, int p0, int np,
                            float *L, cudaStream_t st);
cudaError_t launch_count(const GridDev &g, const ProjGeom *geo, const float2 *trig,
                         int p0, int np, unsigned long long *counts, TileShape ts,
                         cudaStream_t st);
cudaError_t launch_log(const void *in, cyl_dtype it, double i0, void *out, cyl_dtype ot,
                       int64_t n, cudaStream_t st);
cudaError_t launch_convert(const void *in, cyl_dtype it, void *out, cyl_dtype ot,
                           int64_t n, cudaStream_t st);
cudaError_t launch_weight_scale(const float *w, int64_t n, int mode, float lambda,
                                float *wscale, cudaStream_t st);

size_t dtype_size(cyl_dtype t);

}  // namespace cylct
