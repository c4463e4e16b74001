// Stored segment records of a pose.  Every SART subset of every sweep needs each ray's
// row of the system matrix of Eq. 6 twice (the projection q_j = sum_l t_jl x_l, then the
// back-projection of the residual), and the rows depend only on the pose.  Instead of
// walking each ray twice per subset, the walk runs once per pose and writes the row as
// records that the subsets replay: the crossing arithmetic (a square root or a division
// and a three-way comparison per piece) leaves the subsets, which then cost one
// coalesced record load, one gather or reduction and a few integer operations per piece.
//
// A record is 4 bytes: the piece's length t_jl in FP32 with its three lowest mantissa
// bits replaced by the move from the piece's voxel to the next piece's voxel, one of
// eight: shell +-1, wedge +-1, a wedge step across wedge 0 either way, slab +-1.  The
// length is rounded to 20 mantissa bits (relative error <= 2^-21).  A task is 32
// consecutive pixels of one detector row of one view.  Its records are rows of 32 words,
// row s holding piece s of every ray, so a row is one coalesced 128-byte load; a task
// has as many rows as its longest ray has pieces.  The rows are cut into P runs of equal
// length, replayed by the P warps of a block side by side: at every step the 32 lanes of
// a warp touch the voxels of 32 neighbouring rays.  Each ray keeps its piece count and
// the voxel it is in at the first row of every run.
//
// The column sums of Eq. 7 depend on the pose and the subsets only: they are summed once
// per pose (k_rec_den: each view's few pieces per voxel in FP32, the views of a subset in
// FP64) and kept as reciprocals, so the subsets reduce the numerator alone, into one
// 4-byte accumulator that the update clears.
//
// The count walk and the record walk are one kernel (k_rec_walk) in two modes, so both
// produce the same pieces; the record walk checks the count and reports a mismatch.
#include <algorithm>
#include <type_traits>

#include "records.cuh"

namespace cylct {

// mode 0: count the steps of every ray into cnt.  mode 1: write the records at their
// task's rows (row s, lane pixel % 32) and, for every run of ch = ceil(rows / P) rows of
// the task, the voxel the ray is in at the run's first row into idx0 ([ray][P]); a ray
// whose walk gives another count than mode 0 sets *bad.  One thread per ray.
__global__ void __launch_bounds__(256)
k_rec_walk(ScanDev sd, int64_t n_rays, int lgP, int mode, uint32_t *cnt, const int64_t *__restrict__ row_off,
           uint32_t *rec, int32_t *idx0, int *bad)
{
    extern __shared__ float2 s_trig[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig);
    const GridDev &g = sd.g;
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const RayRec rr = ray_at(sd, ray);
    if (!(rr.c.y > rr.c.x)) {
        if (mode == 0) cnt[ray] = 0;
        return;
    }
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int64_t p = ray / npix, pix = ray - p * npix;
    const int64_t task = p * ((npix + 31) >> 5) + (pix >> 5);
    int d[kRecMoves];
    move_deltas(g.n_t, g.n_r, d);
    const uint32_t c = mode == 0 ? 0xffffffffu : cnt[ray];
    const int64_t rows = mode == 0 ? 0 : row_off[task + 1] - row_off[task];
    const int64_t ch = (rows + (1 << lgP) - 1) >> lgP;
    uint32_t *out = mode == 0 ? nullptr : rec + row_off[task] * 32 + (pix & 31);
    Walker wk;
    wk.init(g, s_trig, rr, rr.c.x, rr.c.y);
    int64_t s = 0, run_row = 0, run = 0;   // step; its row within its run; its run
    int pidx = 0;
    float plen = 0.f;
    auto op = [&](int idx, float len) {
        if (out) {
            if (s > 0 && s <= rows) __stcs(out + (s - 1) * 32, rec_encode(plen, move_code(idx - pidx, d)));
            if (run_row == 0 && run < (1 << lgP)) idx0[(ray << lgP) + run] = idx;
            if (++run_row == ch) {
                run_row = 0;
                ++run;
            }
        }
        pidx = idx;
        plen = len;
        ++s;
    };
    while (wk.step(g, s_trig, op)) {
    }
    if (mode == 0) {
        cnt[ray] = (uint32_t)s;
        return;
    }
    if (s >= 1 && s <= rows) __stcs(out + (s - 1) * 32, rec_encode(plen, 0u));
    if ((uint32_t)s != c) atomicOr(bad, 1);
}

// rows of each task: the most pieces among its 32 rays
__global__ void __launch_bounds__(256)
k_rec_rows(const uint32_t *__restrict__ cnt, int64_t npix, int64_t n_tasks, int64_t tpv, int64_t *rows)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_tasks) return;   // the 32 lanes of a warp share w
    const int64_t p = w / tpv, pix = ((w - p * tpv) << 5) + lane;
    const uint32_t c = pix < npix ? cnt[p * npix + pix] : 0u;
    const uint32_t m = __reduce_max_sync(0xffffffffu, c);
    if (lane == 0) rows[w] = m;
}

// Exclusive scan of v[0 .. n) in place by one block of 1024 threads; v[n] = the total.
__global__ void __launch_bounds__(1024) k_rec_scan(int64_t *v, int64_t n)
{
    __shared__ int64_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(a + per, n);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += v[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int64_t x = part[t];
            part[t] = run;
            run += x;
        }
        v[n] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        const int64_t x = v[i];
        v[i] = run;
        run += x;
    }
}

// Column sums of Eq. 7 over one view (tasks [t0, t0 + n_task)): den_m = sum_j t_jm.  One
// warp per run of a task, as the subsets replay them: the 32 rays side by side, the
// pieces of a lane that fall in one aligned quad of voxels going out as one 4 x FP32
// reduction.  A voxel meets about two pieces of a view, each length rounded to 20
// mantissa bits, so these FP32 sums are exact unless the lengths differ by more than a
// factor of 16 (then within 2^-24 relative); the views of a subset add in FP64.
__global__ void __launch_bounds__(256) k_rec_den(RecDev rd, int64_t t0, int64_t n_task, float *den)
{
    __shared__ int s_d[kRecMoves];
    if (threadIdx.x < kRecMoves) s_d[threadIdx.x] = rd.delta[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, lgP = rd.lgP, P = 1 << lgP;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5, n_items = n_task << lgP;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += nw) {
        const int64_t w = t0 + (it >> lgP);
        const int k = (int)(it & (P - 1));
        const int64_t r0 = __ldg(rd.row_off + w), n_rows = __ldg(rd.row_off + w + 1) - r0;
        const int64_t ch = (n_rows + P - 1) >> lgP, a = k * ch;
        const int64_t p = w / rd.tpv, pix = ((w - p * rd.tpv) << 5) + lane;
        const int64_t ray = p * rd.npix + pix;
        const int64_t c = pix < rd.npix ? (int64_t)__ldg(rd.cnt + ray) : 0;
        const int64_t b = min(a + ch, c);
        if (b > a) {   // per lane; the warp takes its next item together
            int idx = __ldg(rd.idx0 + (ray << lgP) + k);
            const uint32_t *rp = rd.rec + r0 * 32 + lane;
            int qc = -1;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
            for (int64_t s = a; s < b; ++s) {
                const uint32_t v = __ldcs(rp + s * 32);
                const float len = rec_len(v);
                const int qn = idx >> 2, sl = idx & 3;
                const bool flush = qn != qc;
                red_add4f_if(flush && qc >= 0, den + 4 * (qc < 0 ? 0 : qc), a0, a1, a2, a3);
                a0 = (flush ? 0.f : a0) + (sl == 0 ? len : 0.f);
                a1 = (flush ? 0.f : a1) + (sl == 1 ? len : 0.f);
                a2 = (flush ? 0.f : a2) + (sl == 2 ? len : 0.f);
                a3 = (flush ? 0.f : a3) + (sl == 3 ? len : 0.f);
                qc = qn;
                idx += s_d[v & 7u];
            }
            red_add4f_if(qc >= 0, den + 4 * (qc < 0 ? 0 : qc), a0, a1, a2, a3);
        }
        __syncwarp();
    }
}

// den64 += den32 (a view of a subset of several views)
__global__ void k_rec_acc(int64_t n, const float *__restrict__ den32, double *__restrict__ den64)
{
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
        den64[m] += (double)__ldg(den32 + m);
}

__device__ __forceinline__ float rec_inv1(float d, float eps) { return d > 0.f ? 1.f / fmaxf(d, eps) : 0.f; }

// r_m = 1 / max(den_m, eps) where den_m > 0, else 0 (the voxel keeps its value in Eq. 7),
// four voxels per thread, from den32 (one view) or den64 (the subset's views added in
// FP64, rounded to FP32 first: FP64 division is slow on this GPU, and r is FP32).  The
// caller clears the sums afterwards.
__global__ void k_rec_inv4(int64_t n4, const float4 *__restrict__ den32, const double2 *__restrict__ den64,
                           float eps, float4 *__restrict__ r)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 d;
        if (den64) {
            const double2 a = __ldg(den64 + 2 * i), b = __ldg(den64 + 2 * i + 1);
            d = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        } else {
            d = __ldg(den32 + i);
        }
        r[i] = make_float4(rec_inv1(d.x, eps), rec_inv1(d.y, eps), rec_inv1(d.z, eps), rec_inv1(d.w, eps));
    }
}

// One SART subset (Eq. 7) from the records: tasks [t0, t0 + n_task) of the pose, one
// task per block of P warps.  Warp k replays run k (rows k ch .. (k + 1) ch - 1) of the
// task's 32 rays side by side, so the lanes of a warp gather and reduce at neighbouring
// voxels: forward, adding t_jl x_l (compensated); the block adds the P runs' sums of each
// ray in FP64 and every warp forms the residual r_j = (p_j - q_j) / max(L_j, eps); each
// warp then replays its run again to back-project r_j into the numerator of Eq. 7 (the
// column sums are the pose's, computed once by k_rec_den): consecutive pieces in one
// aligned quad of voxels go out as one 4 x FP32 reduction.  y holds the launch's views
// from the first task's view on.  sched[0] hands out tasks to blocks; sched[1] counts
// the blocks that found none left, and the last resets both.
// Without BACK (the gather path, gather.cu) the kernel stops after the forward replay and
// writes each ray's residual r_j to resid (the launch's views from the first one on); its
// records are then read once per subset and loaded evict-first (with BACK the backward
// replay reads them again, from L1 or L2).
template <class T, class S, bool BACK>
__global__ void __launch_bounds__(1024)
k_rec_sart(RecDev rd, int64_t t0, int64_t n_task, const T *__restrict__ x, const S *__restrict__ y, float *num,
           float *resid, int *sched)
{
    extern __shared__ double s_q[];          // [P][32] run sums
    __shared__ int s_d[kRecMoves];
    __shared__ int s_f;
    if (threadIdx.x < kRecMoves) s_d[threadIdx.x] = rd.delta[threadIdx.x];
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5, lgP = rd.lgP, P = 1 << lgP;
    const int64_t span = task_span(n_task), p_first = t0 / rd.tpv;
    for (;;) {
        if (threadIdx.x == 0) s_f = atomicAdd(sched, 1);
        __syncthreads();
        const int f = s_f;
        __syncthreads();
        if (f >= span) break;
        const int64_t tt = task_of(f, n_task);
        if (tt < 0) continue;
        const int64_t w = t0 + tt;
        const int64_t r0 = __ldg(rd.row_off + w), n_rows = __ldg(rd.row_off + w + 1) - r0;
        if (n_rows == 0) continue;
        const int64_t ch = (n_rows + P - 1) >> lgP, a = k * ch;
        const int64_t p = w / rd.tpv, pix = ((w - p * rd.tpv) << 5) + lane;
        const int64_t ray = p * rd.npix + pix;
        const int64_t c = pix < rd.npix ? (int64_t)__ldg(rd.cnt + ray) : 0;
        const int64_t b = min(a + ch, c);    // this lane's steps of run k: a .. b - 1
        const int start = b > a ? __ldg(rd.idx0 + (ray << lgP) + k) : 0;
        const uint32_t *rp = rd.rec + r0 * 32 + lane;
        // forward: this run's part of q_j
        int idx = start;
        float acc = 0.f, comp = 0.f;
#pragma unroll 4
        for (int64_t s = a; s < b; ++s) {
            const uint32_t v = BACK ? __ldg(rp + s * 32) : __ldcs(rp + s * 32);
            const float yv = fmaf(rec_len(v), as_f32<T>(__ldg(x + idx)), -comp);
            const float t = acc + yv;
            comp = (t - acc) - yv;
            acc = t;
            idx += s_d[v & 7u];
        }
        s_q[k * 32 + lane] = (double)acc - (double)comp;
        __syncwarp();
        __syncthreads();
        double q = 0.0;
        for (int j = 0; j < P; ++j) q += s_q[j * 32 + lane];
        if (!BACK && k == 0 && c > 0) {   // the gather path back-projects per voxel
            const float L = __ldg(reinterpret_cast<const float *>(rd.ray_c + ray) + 2);
            resid[(p - p_first) * rd.npix + pix] =
                L > 0.f ? (float)(((double)as_f32<S>(y[(p - p_first) * rd.npix + pix]) - q) / fmaxf(L, rd.eps)) : 0.f;
        }
        if (BACK && b > a) {   // per lane; every lane of the block reaches the next fetch's barrier
            const float L = __ldg(reinterpret_cast<const float *>(rd.ray_c + ray) + 2);
            const float yv =
                L > 0.f ? (float)(((double)as_f32<S>(y[(p - p_first) * rd.npix + pix]) - q) / fmaxf(L, rd.eps)) : 0.f;
            // backward: t_jl r_j into num, one reduction per visit of an aligned quad; the
            // run's records are read again, most of them from L1 or L2
            idx = start;
            int qc = -1;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
            for (int64_t s = a; s < b; ++s) {
                const uint32_t v = __ldg(rp + s * 32);
                const float av = rec_len(v) * yv;
                const int qn = idx >> 2, sl = idx & 3;
                const bool flush = qn != qc;
                red_add4f_if(flush && qc >= 0, num + 4 * (qc < 0 ? 0 : qc), a0, a1, a2, a3);
                a0 = (flush ? 0.f : a0) + (sl == 0 ? av : 0.f);
                a1 = (flush ? 0.f : a1) + (sl == 1 ? av : 0.f);
                a2 = (flush ? 0.f : a2) + (sl == 2 ? av : 0.f);
                a3 = (flush ? 0.f : a3) + (sl == 3 ? av : 0.f);
                qc = qn;
                idx += s_d[v & 7u];
            }
            red_add4f_if(qc >= 0, num + 4 * (qc < 0 ? 0 : qc), a0, a1, a2, a3);
        }
        __syncwarp();
    }
    if (threadIdx.x == 0 && (unsigned)atomicAdd(sched + 1, 1) == gridDim.x - 1) {
        atomicExch(sched, 0);
        atomicExch(sched + 1, 0);
    }
}

// Eq. 7's update from the numerator and the pose's reciprocal column sums r:
// x_m += s w_m num_m r_m (r_m = 0 where den_m = 0), then num_m = 0 for the next subset.
// Four voxels per thread with 16-byte accesses (FP32 iterate, aligned arrays, voxel count
// a multiple of 4).
__global__ void k_update_rec4(int64_t n4, float4 *num, const float4 *__restrict__ r, UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    float4 *x = reinterpret_cast<float4 *>(u.x32);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 nv = num[i], rv = __ldg(r + i), wv = weight4_at(u, i);
        float4 xv = x[i];
        xv.x = fmaf(sc * wv.x, nv.x * rv.x, xv.x);
        xv.y = fmaf(sc * wv.y, nv.y * rv.y, xv.y);
        xv.z = fmaf(sc * wv.z, nv.z * rv.z, xv.z);
        xv.w = fmaf(sc * wv.w, nv.w * rv.w, xv.w);
        if (u.clamp) {
            xv.x = rv.x > 0.f ? fmaxf(xv.x, 0.f) : xv.x;
            xv.y = rv.y > 0.f ? fmaxf(xv.y, 0.f) : xv.y;
            xv.z = rv.z > 0.f ? fmaxf(xv.z, 0.f) : xv.z;
            xv.w = rv.w > 0.f ? fmaxf(xv.w, 0.f) : xv.w;
        }
        x[i] = xv;
        num[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// the same per voxel, for every iterate form (FP32, FP32 with a 16-bit copy, 16-bit)
template <class X>
__global__ void k_update_rec(int64_t n, float *num, const float *__restrict__ r, UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    X *x16 = static_cast<X *>(u.x16);
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const float nv = num[m], rv = __ldg(r + m);
        num[m] = 0.f;
        if (rv > 0.f) {
            float xv = u.strict16 ? as_f32<X>(x16[m]) : u.x32[m];
            xv = fmaf(sc * weight_at(u, m), nv * rv, xv);
            if (u.clamp) xv = fmaxf(xv, 0.f);
            if (!u.strict16) u.x32[m] = xv;
            if (x16) x16[m] = from_f32r<X>(xv);
        }
    }
}

// ------------------------------------------------------------------ launchers

template <class F>
static cudaError_t rec_dispatch(cyl_dtype t, F &&f)
{
    switch (t) {
    case CYL_F32: return f((float *)nullptr);
    case CYL_F16: return f((__half *)nullptr);
    case CYL_BF16: return f((__nv_bfloat16 *)nullptr);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rec_rows(const ScanDev &sd, int n_proj, const uint32_t *cnt, int64_t *row_off, cudaStream_t st)
{
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const int64_t tpv = (npix + 31) >> 5, n_tasks = (int64_t)n_proj * tpv;
    if (n_tasks <= 0) return cudaSuccess;
    k_rec_rows<<<(unsigned)((n_tasks + 7) / 8), 256, 0, st>>>(cnt, npix, n_tasks, tpv, row_off);
    k_rec_scan<<<1, 1024, 0, st>>>(row_off, n_tasks);
    return cudaGetLastError();
}

cudaError_t launch_rec_count(const ScanDev &sd, int n_proj, int lgP, uint32_t *cnt, int64_t *row_off,
                             cudaStream_t st)
{
    const int64_t n_rays = (int64_t)n_proj * sd.g.det_w * sd.g.det_h;
    if (n_rays <= 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)sd.g.n_t;
    k_rec_walk<<<(unsigned)((n_rays + 255) / 256), 256, smem, st>>>(sd, n_rays, lgP, 0, cnt, nullptr, nullptr,
                                                                     nullptr, nullptr);
    return launch_rec_rows(sd, n_proj, cnt, row_off, st);
}

cudaError_t launch_rec_fill(const ScanDev &sd, int n_proj, int lgP, uint32_t *cnt, const int64_t *row_off,
                            uint32_t *rec, int32_t *idx0, int *bad, cudaStream_t st)
{
    const int64_t n_rays = (int64_t)n_proj * sd.g.det_w * sd.g.det_h;
    if (n_rays <= 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)sd.g.n_t;
    k_rec_walk<<<(unsigned)((n_rays + 255) / 256), 256, smem, st>>>(sd, n_rays, lgP, 1, cnt, row_off, rec, idx0,
                                                                     bad);
    return cudaGetLastError();
}

RecDev rec_dev(const ScanDev &sd, int lgP, const uint32_t *rec, const int64_t *row_off, const uint32_t *cnt,
               const int32_t *idx0)
{
    RecDev rd;
    rd.rec = rec;
    rd.row_off = row_off;
    rd.cnt = cnt;
    rd.idx0 = idx0;
    rd.ray_c = sd.ray_c;
    rd.npix = (int64_t)sd.g.det_w * sd.g.det_h;
    rd.lgP = lgP;
    rd.tpv = (rd.npix + 31) >> 5;
    move_deltas(sd.g.n_t, sd.g.n_r, rd.delta);
    rd.eps = sd.g.eps;
    return rd;
}

cudaError_t launch_rec_sart(const RecDev &rd, int p0, int np, const void *x, cyl_dtype xt, const void *y,
                            cyl_dtype yt, float *num, float *resid, int *sched, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    // a launch counts its fetches in 32 bits
    const int vmax = (int)std::max<int64_t>(1, ((int64_t)1 << 30) / rd.tpv);
    for (int c0 = 0; c0 < np; c0 += vmax) {
        const int cn = std::min(vmax, np - c0);
        const int64_t t0 = (int64_t)(p0 + c0) * rd.tpv, n_task = (int64_t)cn * rd.tpv;
        const cudaError_t e = rec_dispatch(xt, [&](auto *tx) {
            using T = std::remove_pointer_t<decltype(tx)>;
            return rec_dispatch(yt, [&](auto *ty) {
                using S = std::remove_pointer_t<decltype(ty)>;
                const S *yc = static_cast<const S *>(y) + (int64_t)c0 * rd.npix;
                const int threads = 32 << rd.lgP;
                const size_t smem = sizeof(double) * (size_t)threads;
                float *rc = resid ? resid + (int64_t)c0 * rd.npix : nullptr;
                auto go = [&](auto kern) {
                    const unsigned blocks = persistent_blocks((const void *)kern, smem, 0, threads);
                    kern<<<blocks, threads, smem, st>>>(rd, t0, n_task, (const T *)x, yc, num, rc, sched);
                    return cudaGetLastError();
                };
                return resid ? go(k_rec_sart<T, S, false>) : go(k_rec_sart<T, S, true>);
            });
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_rec_inv_den(const RecDev &rd, int p0, int np, int64_t n_vox, float *den32, double *den64,
                               float *r, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const int64_t n4 = (n_vox + 3) / 4;
    const unsigned ve = (unsigned)std::min<int64_t>((n4 + 255) / 256, 152 * 8);
    for (int v = 0; v < np; ++v) {
        const int64_t t0 = (int64_t)(p0 + v) * rd.tpv;
        const unsigned blocks = (unsigned)std::min<int64_t>(((rd.tpv << rd.lgP) + 7) / 8, 152 * 8);
        k_rec_den<<<blocks, 256, 0, st>>>(rd, t0, rd.tpv, den32);
        if (np > 1) {
            k_rec_acc<<<ve, 256, 0, st>>>(n_vox, den32, den64);
            const cudaError_t e = cudaMemsetAsync(den32, 0, sizeof(float) * 4 * n4, st);
            if (e != cudaSuccess) return e;
        }
    }
    // r and the sums are padded to 4 ceil(V / 4) entries, the pad zero: its r entries are 0
    k_rec_inv4<<<ve, 256, 0, st>>>(n4, reinterpret_cast<const float4 *>(den32),
                                   np > 1 ? reinterpret_cast<const double2 *>(den64) : nullptr, rd.eps,
                                   reinterpret_cast<float4 *>(r));
    const cudaError_t e = np > 1 ? cudaMemsetAsync(den64, 0, sizeof(double) * 4 * n4, st)
                                 : cudaMemsetAsync(den32, 0, sizeof(float) * 4 * n4, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_update_rec(int64_t n_vox, float *num, const float *r, const UpdateArgs &u, cudaStream_t st)
{
    const auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const uintptr_t wb = u.w_t == CYL_F32 ? 16 : (u.w_t == CYL_U8 ? 4 : 8);
    const int64_t blocks = std::min<int64_t>((n_vox / 4 + 255) / 256, 152 * 8);
    if (!u.x16 && !u.strict16 && (n_vox & 3) == 0 && al(u.x32) && al(num) && al(r) &&
        ((uintptr_t)u.w & (wb - 1)) == 0) {
        k_update_rec4<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
            n_vox / 4, reinterpret_cast<float4 *>(num), reinterpret_cast<const float4 *>(r), u);
        return cudaGetLastError();
    }
    const cyl_dtype xt = u.x16 ? u.x16_t : CYL_F32;
    const unsigned b1 = (unsigned)std::max<int64_t>(std::min<int64_t>((n_vox + 255) / 256, 152 * 8), 1);
    return rec_dispatch(xt, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update_rec<X><<<b1, 256, 0, st>>>(n_vox, num, r, u);
        return cudaGetLastError();
    });
}

}  // namespace cylct
