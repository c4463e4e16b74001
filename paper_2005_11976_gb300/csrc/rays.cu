// Ray-driven kernels of Eq. 7.  Every ray is cut into pieces that hold equal numbers of
// steps (the cuts are found once per pose by walking each ray, k_split), and every piece
// is one task for one thread.  The warps of a persistent grid take 32 tasks at a time
// from a work counter.  The long walks of rays through the middle of the grid, where the
// wedge crossings of a ray bunch up around its closest approach to the axis, are thereby
// spread over many threads, and a launch ends when its work ends.  Consecutive fetches
// are sent to kStride parts of the detector far apart (task_of), so the rays in flight
// at any time cover the whole view and their atomics spread over the whole volume.
//   forward:  q_j = sum over the ray of t_jl x_l.  A warp task is ray-major: the P
//             pieces of a ray sit in P adjacent lanes, which add their sums with
//             shuffles; one lane stores q_j (no atomics, no zeroing of q).
//   backward: nd_l += (t_jl r_j, t_jl), a packed 2 x FP32 reduction per segment (the
//             numerator and the column sum of Eq. 7 together), r_j = (p_j - q_j) / L_j;
//             two consecutive segments in the two halves of one 16-byte voxel pair go
//             out as one 4 x FP32 reduction.  A single scan's warp task is ray-major
//             too: with the default P = 2, 16 adjacent rays whose reductions land on
//             neighbouring voxels, each walked by two lanes over halves of equal step
//             counts (the lanes' walks end closer together than those of 32 whole-ray
//             pieces).  Batched rounds keep piece-major tasks (see round_prefix).
//   update:   x_l += s w_l num_l / den_l where den_l > 0 (Eq. 7), elementwise
// The forward kernel also clears the spare accumulator (the one the previous subset's
// update has consumed), so no separate memset pass is needed.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "device_common.cuh"

namespace cylct {

// ------------------------------------------------------------------ piece walks

// Sum of t_jl x_l over a piece, compensated (Kahan): the rounding error of each addition
// is carried into the next, so the sum keeps FP32 accuracy over any number of segments.
// The residual p_j - q_j of a nearly fitted ray cancels most of q_j, which would magnify
// a plainly accumulated sum's rounding.
template <class T>
__device__ __forceinline__ float fp_walk(const GridDev &g, const float2 *__restrict__ trig,
                                         const RayRec &rr, float ua, float ub, const T *__restrict__ x)
{
    Walker w;
    w.init(g, trig, rr, ua, ub);
    float acc = 0.f, comp = 0.f;
    auto op = [&](int idx, float len) {
        const float y = fmaf(len, as_f32<T>(__ldg(x + idx)), -comp);
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    };
    while (w.step(g, trig, op)) {
    }
    return acc - comp;
}

// yv: the ray's value (residual or data); into nd, or into num / den when nd is null
__device__ __forceinline__ void bp_walk(const GridDev &g, const float2 *__restrict__ trig,
                                        const RayRec &rr, float ua, float ub, float yv, float2 *nd,
                                        float *num, float *den)
{
    Walker w;
    w.init(g, trig, rr, ua, ub);
    if (nd) {
        // a segment waits one step: if the next one lands in the other half of the same
        // 16-byte voxel pair (idx ^ pidx == 1; never with pidx = -1), both go out as one
        // 4 x FP32 reduction.  A zero-length segment (a tie of two crossings) adds zeros.
        int pidx = -1;
        float pa = 0.f, pl = 0.f;
        auto op = [&](int idx, float len) {
            const float a = len * yv;
            const bool pair = (idx ^ pidx) == 1;
            const bool lo = (idx & 1) == 0;
            red_add4_if(pair, nd + (idx & ~1), lo ? a : pa, lo ? len : pl, lo ? pa : a, lo ? pl : len);
            red_add2_if(!pair && pidx >= 0, nd + (pidx < 0 ? 0 : pidx), pa, pl);
            pidx = pair ? -1 : idx;
            pa = a;
            pl = len;
        };
        while (w.step(g, trig, op)) {
        }
        red_add2_if(pidx >= 0, nd + (pidx < 0 ? 0 : pidx), pa, pl);
    } else {
        auto op = [&](int idx, float len) {
            if (len > 0.f) {
                atomicAdd(num + idx, len * yv);
                if (den) atomicAdd(den + idx, len);
            }
        };
        while (w.step(g, trig, op)) {
        }
    }
}

// sum over the P adjacent lanes of a ray (P divides 32), in FP64
__device__ __forceinline__ double ray_sum(float v, int P)
{
    double d = v;
    for (int o = P >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    return d;
}

template <class X>
__device__ __forceinline__ void update_voxel(const UpdateArgs &u, int64_t m, float2 v, float sc)
{
    if (!(v.y > 0.f)) return;
    X *x16 = static_cast<X *>(u.x16);
    float xv = u.strict16 ? as_f32<X>(x16[m]) : u.x32[m];
    const float wm = weight_at(u, m);
    xv = fmaf(sc * wm, v.x / fmaxf(v.y, u.den_eps), xv);
    if (u.clamp) xv = fmaxf(xv, 0.f);
    if (!u.strict16) u.x32[m] = xv;
    if (x16) x16[m] = from_f32r<X>(xv);
}

// ------------------------------------------------------------------ set-up

// Steps of a ray's walk, estimated from the crossings of each family between u_in and
// u_out (shells from the radii at both ends and at the closest approach, wedges from the
// angle swept, slabs from the height travelled).
__device__ __forceinline__ float estimate_steps(const GridDev &g, const RayRec &rr)
{
    const float ex = rr.b.x, ey = rr.b.y, d2 = rr.b.w, u0 = rr.c.x, u1 = rr.c.y;
    float n = 1.f + (u1 - u0) * fabsf(rr.b.z) * g.inv_dh;
    if (ray_kstar(rr) >= 0) {
        const float a = fmaf(ex, ex, ey * ey);
        const float r0 = sqrtf(fmaf(a * u0, u0, d2)), r1 = sqrtf(fmaf(a * u1, u1, d2)), rd = sqrtf(d2);
        n += ((u0 < 0.f && u1 > 0.f) ? (r0 - rd) + (r1 - rd) : fabsf(r1 - r0)) * g.inv_dr;
        if (g.n_t > 1) {
            const float x0 = fmaf(u0, ex, rr.a.x), y0 = fmaf(u0, ey, rr.a.y);
            const float x1 = fmaf(u1, ex, rr.a.x), y1 = fmaf(u1, ey, rr.a.y);
            n += fabsf(atan2f(x0 * y1 - y0 * x1, x0 * x1 + y0 * y1)) * g.inv_dth;
        }
    }
    return n;
}

// One thread per ray of every view: walk the ray once and record kSplit - 1 cuts, cut i
// in the middle of the segment that holds step ceil(i N / kSplit) of an estimated N.  The
// last entry keeps the estimate (saturated), for diagnostics.  cnt (if not null) receives
// the ray's number of pieces (the stored segment records are sized from it).
__global__ void __launch_bounds__(256) k_split(ScanDev sd, int64_t n_rays, uint16_t *split, uint32_t *cnt)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_rays) return;
    const RayRec rr = ray_at(sd, j);
    uint16_t *out = split + j * kSplit;
    if (!(rr.c.y > rr.c.x)) {
        for (int i = 0; i < kSplit; ++i) out[i] = 0;
        if (cnt) cnt[j] = 0;
        return;
    }
    const GridDev &g = sd.g;
    const float n_est = estimate_steps(g, rr);
    const float per = n_est / kSplit;
    const float scale = 65535.f / (rr.c.y - rr.c.x);
    Walker w;
    w.init(g, sd.trig, rr, rr.c.x, rr.c.y);
    int s = 0, next = 1;
    auto op = [&](int, float len) {
        ++s;
        while (next < kSplit && (float)s >= ceilf(next * per)) {
            const float f = (fmaf(0.5f, len, w.u) - rr.c.x) * scale;
            out[next - 1] = (uint16_t)fminf(fmaxf(f, 0.f), 65535.f);
            ++next;
        }
    };
    while (w.step(g, sd.trig, op)) {
    }
    for (; next < kSplit; ++next) out[next - 1] = 65535;
    out[kSplit - 1] = (uint16_t)fminf(n_est, 65535.f);
    if (cnt) cnt[j] = (uint32_t)s;
}

// ------------------------------------------------------------------ listed rays

// A compact plan keeps, per pose, only the rays of positive chord (u_out > u_in): listed
// view by view in ray order, with their records and cuts stored at their list positions.
// Each block sets up one chunk of kActChunk rays of one view (FP64, setup_ray) and counts
// the ones that meet the grid; one block scans the chunk counts; the fill pass sets the
// chunk up again and writes each listed ray's index and record at its position (ranks
// from warp ballots).
__global__ void __launch_bounds__(256) k_act_count(GridDev g, const ProjGeom *__restrict__ geo, int cpv,
                                                   int64_t *chunk)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int64_t p = blockIdx.y, j0 = (int64_t)blockIdx.x * kActChunk;
    int n = 0;
    for (int k = threadIdx.x; k < kActChunk; k += blockDim.x) {
        const int64_t j = j0 + k;
        bool on = false;
        if (j < npix) {
            const RayRec rr = setup_ray(g, geo[p], (int)(j % g.det_w), (int)(j / g.det_w));
            on = rr.c.y > rr.c.x;
        }
        n += __syncthreads_count(on);
    }
    if (threadIdx.x == 0) chunk[p * cpv + blockIdx.x] = n;
}

// Exclusive scan of the chunk counts in place (one block of 1024 threads), then the
// per-view offsets: act_off[p] = offset of view p's first chunk, act_off[n_proj] = total.
__global__ void __launch_bounds__(1024) k_act_scan(int64_t *chunk, int64_t n, int n_proj, int cpv, int64_t *act_off)
{
    __shared__ int64_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(a + per, n);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += chunk[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int64_t v = part[t];
            part[t] = run;
            run += v;
        }
        act_off[n_proj] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        const int64_t v = chunk[i];
        chunk[i] = run;
        run += v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n_proj; p += blockDim.x) act_off[p] = chunk[(int64_t)p * cpv];
}

// cap: entries the list and record buffers hold (the scan's total, read by the host)
__global__ void __launch_bounds__(256) k_act_fill(GridDev g, const ProjGeom *__restrict__ geo, int cpv,
                                                  const int64_t *chunk, int64_t cap, uint32_t *act, float4 *ra,
                                                  float4 *rb, float4 *rc)
{
    __shared__ int warp_n[8];
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int64_t p = blockIdx.y, j0 = (int64_t)blockIdx.x * kActChunk;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t pos = chunk[p * cpv + blockIdx.x];
    for (int k = 0; k < kActChunk; k += blockDim.x) {
        const int64_t j = j0 + k + threadIdx.x;
        RayRec rr{};
        bool on = false;
        if (j < npix) {
            rr = setup_ray(g, geo[p], (int)(j % g.det_w), (int)(j / g.det_w));
            on = rr.c.y > rr.c.x;
        }
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) warp_n[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < 8; ++q) {
            before += q < w ? warp_n[q] : 0;
            total += warp_n[q];
        }
        const int64_t e = pos + before + __popc(m & ((1u << lane) - 1u));
        if (on && e < cap) {
            act[e] = (uint32_t)(p * npix + j);
            ra[e] = rr.a;
            rb[e] = rr.b;
            rc[e] = rr.c;
        }
        pos += total;
        __syncthreads();
    }
}

// Tasks of a launch over the rays of views p0 .. : with LIST, the launch's part
// [a0, a0 + n_task) of the list of rays of positive chord; else every ray.
template <bool LIST>
__device__ __forceinline__ void launch_tasks(const RayList &rl, int p0, int64_t npix, int64_t n_rays, int64_t &a0,
                                             int64_t &n_task)
{
    a0 = 0;
    n_task = n_rays;
    if (LIST) {
        a0 = rl.act_off[p0];
        n_task = rl.act_off[p0 + n_rays / npix] - a0;
    }
}

// ------------------------------------------------------------------ single scan

// Rays j in [0, n_rays) are rays p0 * H * W + j of the plan; lgP = log2(P).  With LIST
// only the rays of positive chord are tasks and only their q is written.
template <class T, bool LIST>
__global__ void __launch_bounds__(256)
k_fp(ScanDev sd, int lgP, int p0, int64_t n_rays, const T *__restrict__ x, float *__restrict__ q,
     float2 *zero_buf, int64_t zero_len, RayList rl)
{
    extern __shared__ float2 s_trig[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig);
    zero_slice(zero_buf, zero_len, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h, base = (int64_t)p0 * npix;
    int64_t a0, n_task;
    launch_tasks<LIST>(rl, p0, npix, n_rays, a0, n_task);
    const int64_t n_wt = ((n_task << lgP) + 31) >> 5, span = task_span(n_wt);
    for (;;) {
        const int f = fetch_task(sd.sched);
        if (f >= span) break;
        const int64_t wt = task_of(f, n_wt);
        if (wt < 0) continue;
        const int64_t t = wt * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (P - 1));
        float acc = 0.f;
        int64_t r = -1;
        if (i < n_task) {
            // a listed ray's record and cuts sit at its list position
            r = LIST ? (int64_t)__ldg(rl.act + a0 + i) - base : i;
            const int64_t rec = LIST ? a0 + i : base + r;
            const RayRec rr = ray_at(sd, rec);
            float ua, ub;
            if (piece_bounds(rr, sd.split + rec * kSplit, piece, P, ua, ub))
                acc = fp_walk<T>(sd.g, s_trig, rr, ua, ub, x);
        }
        acc = ray_sum(acc, P);
        if (piece == 0 && r >= 0) q[r] = acc;
    }
    retire(sd.sched);
}

// y, q: the launch's rays (indexed like r); SART: residual (y - q) / L, else y
template <class S, bool SART, bool LIST>
__global__ void __launch_bounds__(256)
k_bp(ScanDev sd, int lgP, int p0, int64_t n_rays, const S *__restrict__ y, const float *__restrict__ q,
     float2 *nd, float *num, float *den, RayList rl)
{
    extern __shared__ float2 s_trig[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig);
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h, base = (int64_t)p0 * npix;
    int64_t a0, n_task;
    launch_tasks<LIST>(rl, p0, npix, n_rays, a0, n_task);
    const int64_t n_wt = ((n_task << lgP) + 31) >> 5, span = task_span(n_wt);
    int *sched = sd.sched + 2;
    for (;;) {
        const int f = fetch_task(sched);
        if (f >= span) break;
        const int64_t wt = task_of(f, n_wt);
        if (wt < 0) continue;
        const int64_t t = wt * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (P - 1));
        if (i >= n_task) continue;
        const int64_t r = LIST ? (int64_t)__ldg(rl.act + a0 + i) - base : i;
        const int64_t rec = LIST ? a0 + i : base + r;
        const RayRec rr = ray_at(sd, rec);
        float ua, ub;
        if (!piece_bounds(rr, sd.split + rec * kSplit, piece, P, ua, ub)) continue;
        float yv;
        if (SART) {
            const float L = rr.c.z;
            yv = L > 0.f ? (as_f32<S>(y[r]) - q[r]) / fmaxf(L, sd.g.eps) : 0.f;
        } else {
            yv = as_f32<S>(y[r]);
            if (yv == 0.f && !den) continue;
        }
        bp_walk(sd.g, s_trig, rr, ua, ub, yv, nd, num, den);
    }
    retire(sched);
}

// One SART subset in one launch (Eq. 7).  A warp task holds 32 / P rays, the P pieces
// of a ray in P adjacent lanes.  Each lane walks its piece forward, adding t_jl x_l; the
// P lanes sum q_j and form the residual r_j = (p_j - q_j) / L_j; each lane then walks its
// piece again, back-projecting r_j into the packed (numerator, column sum) accumulator.
// One launch instead of a projector and a back-projector: the projections never go to
// memory, and the gathers of some warps overlap the reductions of others.  The spare
// accumulator is cleared on the way, as in k_fp.
template <class T, class S, bool LIST>
__global__ void __launch_bounds__(kSartThreads)
k_sart(ScanDev sd, int lgP, int p0, int64_t n_rays, const T *__restrict__ x, const S *__restrict__ y, float2 *nd,
       float2 *zero_buf, int64_t zero_len, RayList rl)
{
    extern __shared__ float2 s_trig[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig);
    zero_slice(zero_buf, zero_len, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h, base = (int64_t)p0 * npix;
    int64_t a0, n_task;
    launch_tasks<LIST>(rl, p0, npix, n_rays, a0, n_task);
    const int64_t n_wt = ((n_task << lgP) + 31) >> 5, span = task_span(n_wt);
    int *sched = sd.sched + 6;
    for (;;) {
        const int f = fetch_task(sched);
        if (f >= span) break;
        const int64_t wt = task_of(f, n_wt);
        if (wt < 0) continue;
        const int64_t t = wt * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (P - 1));
        float acc = 0.f, ua = 0.f, ub = 0.f;
        int64_t r = -1, rec = 0;
        bool have = false;
        if (i < n_task) {
            r = LIST ? (int64_t)__ldg(rl.act + a0 + i) - base : i;
            rec = LIST ? a0 + i : base + r;
            const RayRec rr = ray_at(sd, rec);
            have = piece_bounds(rr, sd.split + rec * kSplit, piece, P, ua, ub);
            if (have) acc = fp_walk<T>(sd.g, s_trig, rr, ua, ub, x);
        }
        const double q = ray_sum(acc, P);
        if (!have) continue;
        const RayRec rr = ray_at(sd, rec);
        const float L = rr.c.z;
        const float yv = L > 0.f ? (float)(((double)as_f32<S>(y[r]) - q) / fmaxf(L, sd.g.eps)) : 0.f;
        bp_walk(sd.g, s_trig, rr, ua, ub, yv, nd, nullptr, nullptr);
    }
    retire(sched);
}

// The FP32 iterate without a 16-bit copy: four voxels per thread, 16-byte loads and
// stores (the same arithmetic as update_voxel; voxels with den = 0 keep their value).
__device__ __forceinline__ float upd1(float x, float num, float den, float w, float sc, int clamp, float eps)
{
    if (!(den > 0.f)) return x;
    x = fmaf(sc * w, num / fmaxf(den, eps), x);
    return clamp ? fmaxf(x, 0.f) : x;
}

// voxels 4i .. 4i + 3
__device__ __forceinline__ void update4(const UpdateArgs &u, const float4 *__restrict__ nd, int64_t i, float sc)
{
    float4 *x = reinterpret_cast<float4 *>(u.x32);
    const float4 a = __ldg(nd + 2 * i), b = __ldg(nd + 2 * i + 1);
    const float4 wv = weight4_at(u, i);
    float4 xv = x[i];
    xv.x = upd1(xv.x, a.x, a.y, wv.x, sc, u.clamp, u.den_eps);
    xv.y = upd1(xv.y, a.z, a.w, wv.y, sc, u.clamp, u.den_eps);
    xv.z = upd1(xv.z, b.x, b.y, wv.z, sc, u.clamp, u.den_eps);
    xv.w = upd1(xv.w, b.z, b.w, wv.w, sc, u.clamp, u.den_eps);
    x[i] = xv;
}

__host__ __device__ inline bool update4_ok(const UpdateArgs &u, const void *nd, int64_t n)
{
    const auto al = [](const void *p, uintptr_t b) { return ((uintptr_t)p & (b - 1)) == 0; };
    const uintptr_t wb = u.w_t == CYL_F32 ? 16 : (u.w_t == CYL_U8 ? 4 : 8);
    return !u.x16 && !u.strict16 && (n & 3) == 0 && al(u.x32, 16) && al(u.w, wb) && al(nd, 16);
}

__global__ void k_update_nd4(int64_t n4, const float4 *__restrict__ nd, UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x)
        update4(u, nd, i, sc);
}

template <class X>
__global__ void k_update_nd(int64_t n, const float2 *__restrict__ nd, UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x)
        update_voxel<X>(u, m, __ldg(nd + m), sc);
}

// Segments of positive length per view; a cut inside a segment is not counted twice.
template <bool LIST>
__global__ void __launch_bounds__(256)
k_count(ScanDev sd, int p0, int64_t n_rays, unsigned long long *counts, RayList rl)
{
    extern __shared__ float2 s_trig[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig);
    const int lane = threadIdx.x & 31;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h, base = p0 * npix;
    constexpr int lgP = 4;   // kSplit pieces
    static_assert(kSplit == 1 << lgP, "kSplit is 2^4");
    int64_t a0, n_task;
    launch_tasks<LIST>(rl, p0, npix, n_rays, a0, n_task);
    const int64_t n_wt = ((n_task << lgP) + 31) >> 5;
    int *sched = sd.sched + 4;
    for (;;) {
        const int wt = fetch_task(sched);
        if (wt >= n_wt) break;
        const int64_t t = (int64_t)wt * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (kSplit - 1));
        if (i >= n_task) continue;
        const int64_t r = LIST ? (int64_t)__ldg(rl.act + a0 + i) - base : i;
        const int64_t rec = LIST ? a0 + i : base + r;
        const RayRec rr = ray_at(sd, rec);
        float ua, ub;
        if (!piece_bounds(rr, sd.split + rec * kSplit, piece, kSplit, ua, ub)) continue;
        Walker w;
        w.init(sd.g, s_trig, rr, ua, ub);
        unsigned int n = 0;
        auto op = [&](int, float len) { n += len > 0.f; };
        while (w.step(sd.g, s_trig, op)) {
        }
        if (piece > 0 && n > 0) --n;
        if (n) atomicAdd(counts + r / npix, (unsigned long long)n);
    }
    retire(sched);
}

// ------------------------------------------------------------------ batched rounds

// Warp tasks of the round's items, item-aligned (a warp task never spans two items):
// s_pre[k] = first warp task of item k, s_pre[n] = total.  Thread 0 fills it.  An item
// of `rays` rays has ceil(rays P / 32) ray-major warp tasks (forward) or ceil(rays / 32) P
// piece-major ones (backward: the same piece of 32 adjacent rays; with the rays of many
// scans in flight this measured 1.7 % faster than ray-major tasks at the tuned P = 2).
// rays of item `it` that are tasks, and the first of them in the scan's list
template <bool LIST>
__device__ __forceinline__ int64_t item_rays(const BatchScan &sc, const BatchItem &it, int64_t &a0)
{
    a0 = 0;
    if (LIST && sc.rl.act) {
        a0 = sc.rl.act_off[it.p0];
        return sc.rl.act_off[it.p0 + it.np] - a0;
    }
    return (int64_t)it.np * sc.sd.g.det_w * sc.sd.g.det_h;
}

template <bool PIECE_MAJOR, bool LIST>
__device__ __forceinline__ int round_prefix(const BatchScan *__restrict__ scans,
                                            const BatchItem *__restrict__ its, int n, int lgP,
                                            int *s_pre)
{
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < n; ++k) {
            s_pre[k] = acc;
            const BatchScan &sc = scans[its[k].scan];
            int64_t a0;
            const int64_t rays = item_rays<LIST>(sc, its[k], a0);
            acc += PIECE_MAJOR ? (int)(((rays + 31) >> 5) << lgP) : (int)(((rays << lgP) + 31) >> 5);
        }
        s_pre[n] = acc;
    }
    __syncthreads();
    return s_pre[n];
}

// the item whose warp tasks hold wt (s_pre ascending, n >= 1)
__device__ __forceinline__ int item_of(const int *s_pre, int n, int wt)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= wt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class T, bool LIST>
__global__ void __launch_bounds__(256)
k_fp_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
           const int *__restrict__ n_items, int max_items, int round, int lgP, int *sched)
{
    extern __shared__ int s_pre[];
    const int n = n_items[round];
    const BatchItem *its = items + (int64_t)round * max_items;
    const int total = round_prefix<false, LIST>(scans, its, n, lgP, s_pre);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < n; ++k) {   // spare accumulators of every item's scan
        const BatchScan &sc = scans[its[k].scan];
        zero_slice(sc.nd[its[k].buf ^ 1], sc.nd_len, tid, nth);
    }
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    for (;;) {
        const int wt = fetch_task(sched);
        if (wt >= total) break;
        const int k = item_of(s_pre, n, wt);
        const BatchItem it = its[k];
        const BatchScan &sc = scans[it.scan];
        const int64_t npix = (int64_t)sc.sd.g.det_w * sc.sd.g.det_h;
        const int64_t base = it.p0 * npix;
        int64_t a0;
        const int64_t n_task = item_rays<LIST>(sc, it, a0);
        const int64_t t = (int64_t)(wt - s_pre[k]) * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (P - 1));
        float acc = 0.f;
        int64_t r = -1;
        if (i < n_task) {
            const bool listed = LIST && sc.rl.act;
            r = listed ? (int64_t)__ldg(sc.rl.act + a0 + i) - base : i;
            const int64_t rec = listed ? a0 + i : base + r;
            const RayRec rr = ray_at(sc.sd, rec);
            float ua, ub;
            if (piece_bounds(rr, sc.sd.split + rec * kSplit, piece, P, ua, ub))
                acc = fp_walk<T>(sc.sd.g, sc.sd.trig, rr, ua, ub, static_cast<const T *>(sc.x_proj));
        }
        acc = ray_sum(acc, P);
        if (piece == 0 && r >= 0) sc.q[it.buf][r] = acc;
    }
    retire(sched);
}

template <class S, bool LIST>
__global__ void __launch_bounds__(256)
k_bp_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
           const int *__restrict__ n_items, int max_items, int round, int lgP, int *sched)
{
    extern __shared__ int s_pre[];
    const int n = n_items[round];
    const BatchItem *its = items + (int64_t)round * max_items;
    const int total = round_prefix<true, LIST>(scans, its, n, lgP, s_pre);
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    for (;;) {
        const int wt = fetch_task(sched + 2);
        if (wt >= total) break;
        const int k = item_of(s_pre, n, wt);
        const BatchItem it = its[k];
        const BatchScan &sc = scans[it.scan];
        const int64_t npix = (int64_t)sc.sd.g.det_w * sc.sd.g.det_h;
        const int64_t base = it.p0 * npix;
        int64_t a0;
        const int64_t n_task = item_rays<LIST>(sc, it, a0);
        const int wl = wt - s_pre[k];
        const int64_t i = (int64_t)(wl >> lgP) * 32 + lane;
        const int piece = wl & (P - 1);
        if (i >= n_task) continue;
        const bool listed = LIST && sc.rl.act;
        const int64_t r = listed ? (int64_t)__ldg(sc.rl.act + a0 + i) - base : i;
        const int64_t rec = listed ? a0 + i : base + r;
        const RayRec rr = ray_at(sc.sd, rec);
        float ua, ub;
        if (!piece_bounds(rr, sc.sd.split + rec * kSplit, piece, P, ua, ub)) continue;
        const float L = rr.c.z;
        const S *y = static_cast<const S *>(sc.sino) + base;
        const float yv = L > 0.f ? (as_f32<S>(y[r]) - sc.q[it.buf][r]) / fmaxf(L, sc.sd.g.eps) : 0.f;
        bp_walk(sc.sd.g, sc.sd.trig, rr, ua, ub, yv, sc.nd[it.buf], nullptr, nullptr);
    }
    retire(sched + 2);
}

// One round of a batched solve in one launch per the single-scan k_sart: the round's
// items' rays as ray-major warp tasks, each ray walked forward, its residual formed from
// the lanes' FP64 sum, and walked again to back-project it.
template <class T, class S, bool LIST>
__global__ void __launch_bounds__(256)
k_sart_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
             const int *__restrict__ n_items, int max_items, int round, int lgP, int *sched)
{
    extern __shared__ int s_pre[];
    const int n = n_items[round];
    const BatchItem *its = items + (int64_t)round * max_items;
    const int total = round_prefix<false, LIST>(scans, its, n, lgP, s_pre);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < n; ++k) {   // spare accumulators of every item's scan
        const BatchScan &sc = scans[its[k].scan];
        zero_slice(sc.nd[its[k].buf ^ 1], sc.nd_len, tid, nth);
    }
    const int P = 1 << lgP, lane = threadIdx.x & 31;
    for (;;) {
        const int wt = fetch_task(sched + 6);
        if (wt >= total) break;
        const int k = item_of(s_pre, n, wt);
        const BatchItem it = its[k];
        const BatchScan &sc = scans[it.scan];
        const int64_t npix = (int64_t)sc.sd.g.det_w * sc.sd.g.det_h;
        const int64_t base = it.p0 * npix;
        int64_t a0;
        const int64_t n_task = item_rays<LIST>(sc, it, a0);
        const int64_t t = (int64_t)(wt - s_pre[k]) * 32 + lane, i = t >> lgP;
        const int piece = (int)(t & (P - 1));
        float acc = 0.f, ua = 0.f, ub = 0.f;
        int64_t r = -1, rec = 0;
        bool have = false;
        if (i < n_task) {
            const bool listed = LIST && sc.rl.act;
            r = listed ? (int64_t)__ldg(sc.rl.act + a0 + i) - base : i;
            rec = listed ? a0 + i : base + r;
            const RayRec rr = ray_at(sc.sd, rec);
            have = piece_bounds(rr, sc.sd.split + rec * kSplit, piece, P, ua, ub);
            if (have) acc = fp_walk<T>(sc.sd.g, sc.sd.trig, rr, ua, ub, static_cast<const T *>(sc.x_proj));
        }
        const double q = ray_sum(acc, P);
        if (!have) continue;
        const RayRec rr = ray_at(sc.sd, rec);
        const float L = rr.c.z;
        const S *y = static_cast<const S *>(sc.sino) + base;
        const float yv = L > 0.f ? (float)(((double)as_f32<S>(y[r]) - q) / fmaxf(L, sc.sd.g.eps)) : 0.f;
        bp_walk(sc.sd.g, sc.sd.trig, rr, ua, ub, yv, sc.nd[it.buf], nullptr, nullptr);
    }
    retire(sched + 6);
}

template <class X>
__global__ void k_update_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
                               const int *__restrict__ n_items, int max_items, int round)
{
    const int k = blockIdx.y;
    if (k >= n_items[round]) return;
    const BatchItem it = items[(int64_t)round * max_items + k];
    const BatchScan &sc = scans[it.scan];
    const float sc_ = sc.upd.wscale ? *sc.upd.wscale : sc.upd.lambda;
    const float2 *nd = sc.nd[it.buf];
    if (update4_ok(sc.upd, nd, sc.nd_len)) {
        const float4 *nd4 = reinterpret_cast<const float4 *>(nd);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (sc.nd_len >> 2);
             i += (int64_t)gridDim.x * blockDim.x)
            update4(sc.upd, nd4, i, sc_);
        return;
    }
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < sc.nd_len;
         m += (int64_t)gridDim.x * blockDim.x)
        update_voxel<X>(sc.upd, m, __ldg(nd + m), sc_);
}

// ------------------------------------------------------------------ launchers

template <class F>
static cudaError_t dispatch_t(cyl_dtype t, F &&f)
{
    switch (t) {
    case CYL_F32: return f((float *)nullptr);
    case CYL_F16: return f((__half *)nullptr);
    case CYL_BF16: return f((__nv_bfloat16 *)nullptr);
    }
    return cudaErrorInvalidValue;
}

static inline size_t trig_smem(int n_t) { return sizeof(float2) * (size_t)n_t; }

static inline int update_blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

// log2 of P (P <= 0: the kernel's default); -1 unless P is a power of two dividing kSplit
static int log2_pieces(int P, int dflt)
{
    if (P <= 0) P = dflt;
    int l = 0;
    while ((1 << l) < P) ++l;
    return (1 << l) == P && P <= kSplit ? l : -1;
}

// Resident 256-thread blocks per SM of the back-projectors' persistent grids.  Fewer
// warps in flight than fit (4 by registers) measured faster, the fewer the faster: the
// medium view's k_bp took 97.2 us at 2 blocks, 103 - 105.5 at 3, 111.7 - 113.8 at 4 and
// 131 at 5 (forced to 48 registers); fewer reductions in flight contend less in L2.
// k_fp is fastest with all 5 that fit (78.9 us; 83.2 at 4, 88.6 at 3).  The batched
// back-projector (60 registers, 4 blocks fit) runs at 3: 5.57 vs 5.41 scans/s at 4 for
// a 64-scan batch, and the same at 2.
constexpr int kBpBlocksPerSm = 2, kBpBatchBlocksPerSm = 3;

unsigned persistent_blocks(const void *kernel, size_t smem, int cap, int threads)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, std::pair<int, size_t>>, unsigned> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(kernel, std::make_pair(dev * 4096 + threads, smem));
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n_sm = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        n_sm < 1 || per_sm < 1) {
        cudaGetLastError();
        return 152;
    }
    const unsigned b = (unsigned)(n_sm * (cap > 0 ? std::min(per_sm, cap) : per_sm));
    cache[key] = b;
    return b;
}

int valid_pieces(int P) { return log2_pieces(P, kSplit) >= 0; }
int default_pieces(int kind) { return kind == 0 ? kPiecesFp : kPiecesBp; }

cudaError_t launch_split(const ScanDev &sd, int64_t n_rays, uint16_t *split, cudaStream_t st, uint32_t *cnt)
{
    if (n_rays <= 0) return cudaSuccess;
    k_split<<<(unsigned)((n_rays + 255) / 256), 256, 0, st>>>(sd, n_rays, split, cnt);
    return cudaGetLastError();
}

// A spin of the part about its own axis leaves the grid cylinder, and so the list, as it
// is: only the listed rays' records are set up again.
__global__ void k_act_refill(GridDev g, const ProjGeom *__restrict__ geo, const uint32_t *__restrict__ act,
                             int64_t n, float4 *ra, float4 *rb, float4 *rc)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = act[e], p = j / npix, pix = j - p * npix;
        const RayRec rr = setup_ray(g, geo[p], (int)(pix % g.det_w), (int)(pix / g.det_w));
        ra[e] = rr.a;
        rb[e] = rr.b;
        rc[e] = rr.c;
    }
}

cudaError_t launch_list_refill(const GridDev &g, const ProjGeom *geo, const uint32_t *act, int64_t n, float4 *ra,
                               float4 *rb, float4 *rc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_act_refill<<<(unsigned)blocks, 256, 0, st>>>(g, geo, act, n, ra, rb, rc);
    return cudaGetLastError();
}

cudaError_t launch_list_count(const GridDev &g, const ProjGeom *geo, int n_proj, int64_t *chunk, int64_t *act_off,
                              cudaStream_t st)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int cpv = (int)((npix + kActChunk - 1) / kActChunk);
    if (n_proj <= 0 || npix <= 0) return cudaSuccess;
    k_act_count<<<dim3((unsigned)cpv, (unsigned)n_proj), 256, 0, st>>>(g, geo, cpv, chunk);
    k_act_scan<<<1, 1024, 0, st>>>(chunk, (int64_t)n_proj * cpv, n_proj, cpv, act_off);
    return cudaGetLastError();
}

cudaError_t launch_list_fill(const GridDev &g, const ProjGeom *geo, int n_proj, const int64_t *chunk, int64_t cap,
                             uint32_t *act, float4 *ra, float4 *rb, float4 *rc, cudaStream_t st)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int cpv = (int)((npix + kActChunk - 1) / kActChunk);
    if (n_proj <= 0 || npix <= 0) return cudaSuccess;
    k_act_fill<<<dim3((unsigned)cpv, (unsigned)n_proj), 256, 0, st>>>(g, geo, cpv, chunk, cap, act, ra, rb, rc);
    return cudaGetLastError();
}

// Views per launch: a launch counts its warp tasks in 32 bits (at most H W / 2 per view
// with 16 pieces per ray), so very long view ranges go out as several launches.
static int views_per_launch(const ScanDev &sd)
{
    const int64_t per_view = (int64_t)sd.g.det_w * sd.g.det_h / 2 + 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)1 << 30) / per_view, 1 << 30));
}

cudaError_t launch_fp_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt,
                           float *q, float2 *zero_buf, int64_t zero_len, cudaStream_t st, const RayList &rl)
{
    if (np <= 0) return cudaSuccess;
    const int lgP = log2_pieces(P, kPiecesFp);
    if (lgP < 0) return cudaErrorInvalidValue;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const size_t smem = trig_smem(sd.g.n_t);
    const int vmax = views_per_launch(sd);
    for (int c0 = 0; c0 < np; c0 += vmax) {
        const int cn = std::min(vmax, np - c0);
        const int64_t n_rays = (int64_t)cn * npix;
        float *qc = q + (int64_t)c0 * npix;
        float2 *zb = c0 == 0 ? zero_buf : nullptr;
        const int64_t zl = c0 == 0 ? zero_len : 0;
        const cudaError_t e = dispatch_t(xt, [&](auto *tx) {
            using T = std::remove_pointer_t<decltype(tx)>;
            if (rl.act) {
                const unsigned blocks = persistent_blocks((const void *)k_fp<T, true>, smem);
                k_fp<T, true><<<blocks, 256, smem, st>>>(sd, lgP, p0 + c0, n_rays, (const T *)x, qc, zb, zl, rl);
            } else {
                const unsigned blocks = persistent_blocks((const void *)k_fp<T, false>, smem);
                k_fp<T, false><<<blocks, 256, smem, st>>>(sd, lgP, p0 + c0, n_rays, (const T *)x, qc, zb, zl, rl);
            }
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bp_rays(const ScanDev &sd, int P, int p0, int np, const void *y, cyl_dtype yt,
                           const float *q, float2 *nd, float *num, float *den, cudaStream_t st, const RayList &rl)
{
    if (np <= 0) return cudaSuccess;
    const int lgP = log2_pieces(P, kPiecesBp);
    if (lgP < 0) return cudaErrorInvalidValue;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const size_t smem = trig_smem(sd.g.n_t);
    const int vmax = views_per_launch(sd);
    for (int c0 = 0; c0 < np; c0 += vmax) {
        const int cn = std::min(vmax, np - c0);
        const int64_t n_rays = (int64_t)cn * npix;
        const float *qc = q ? q + (int64_t)c0 * npix : nullptr;
        const cudaError_t e = dispatch_t(yt, [&](auto *ty) {
            using S = std::remove_pointer_t<decltype(ty)>;
            const S *yc = static_cast<const S *>(y) + (int64_t)c0 * npix;
            auto go = [&](auto kern) {
                const unsigned blocks = persistent_blocks((const void *)kern, smem, kBpBlocksPerSm);
                kern<<<blocks, 256, smem, st>>>(sd, lgP, p0 + c0, n_rays, yc, qc, nd, num, den, rl);
            };
            if (qc) {
                if (rl.act) go(k_bp<S, true, true>);
                else go(k_bp<S, true, false>);
            } else {
                if (rl.act) go(k_bp<S, false, true>);
                else go(k_bp<S, false, false>);
            }
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sart_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt, const void *y,
                             cyl_dtype yt, float2 *nd, float2 *zero_buf, int64_t zero_len, cudaStream_t st,
                             const RayList &rl)
{
    if (np <= 0) return cudaSuccess;
    const int lgP = log2_pieces(P, kPiecesSart);
    if (lgP < 0) return cudaErrorInvalidValue;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const size_t smem = trig_smem(sd.g.n_t);
    const int vmax = views_per_launch(sd);
    for (int c0 = 0; c0 < np; c0 += vmax) {
        const int cn = std::min(vmax, np - c0);
        const int64_t n_rays = (int64_t)cn * npix;
        float2 *zb = c0 == 0 ? zero_buf : nullptr;
        const int64_t zl = c0 == 0 ? zero_len : 0;
        const cudaError_t e = dispatch_t(xt, [&](auto *tx) {
            using T = std::remove_pointer_t<decltype(tx)>;
            return dispatch_t(yt, [&](auto *ty) {
                using S = std::remove_pointer_t<decltype(ty)>;
                const S *yc = static_cast<const S *>(y) + (int64_t)c0 * npix;
                auto go = [&](auto kern) {
                    const unsigned blocks = persistent_blocks((const void *)kern, smem, 0, kSartThreads);
                    kern<<<blocks, kSartThreads, smem, st>>>(sd, lgP, p0 + c0, n_rays, (const T *)x, yc, nd, zb, zl,
                                                             rl);
                    return cudaGetLastError();
                };
                return rl.act ? go(k_sart<T, S, true>) : go(k_sart<T, S, false>);
            });
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_update_nd(int64_t n_vox, const float2 *nd, const UpdateArgs &u, cudaStream_t st)
{
    if (update4_ok(u, nd, n_vox)) {
        k_update_nd4<<<update_blocks(n_vox / 4), 256, 0, st>>>(n_vox / 4, reinterpret_cast<const float4 *>(nd), u);
        return cudaGetLastError();
    }
    const cyl_dtype xt = u.x16 ? u.x16_t : CYL_F32;
    return dispatch_t(xt, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update_nd<X><<<update_blocks(n_vox), 256, 0, st>>>(n_vox, nd, u);
        return cudaGetLastError();
    });
}

cudaError_t launch_count_rays(const ScanDev &sd, int p0, int np, unsigned long long *counts, cudaStream_t st,
                              const RayList &rl)
{
    if (np <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const size_t smem = trig_smem(sd.g.n_t);
    const int vmax = views_per_launch(sd);
    for (int c0 = 0; c0 < np; c0 += vmax) {
        const int cn = std::min(vmax, np - c0);
        auto go = [&](auto kern) {
            kern<<<persistent_blocks((const void *)kern, smem), 256, smem, st>>>(sd, p0 + c0, (int64_t)cn * npix,
                                                                                 counts + c0, rl);
        };
        if (rl.act) go(k_count<true>);
        else go(k_count<false>);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_batch_round(const BatchScan *scans, const BatchItem *items, const int *n_items,
                               int max_items, int round, int64_t max_vox, int Pf, int Pb, int parts,
                               int *sched, cyl_dtype xt, cyl_dtype yt, cyl_dtype x16t, cudaStream_t st,
                               bool lists)
{
    const int lgPf = log2_pieces(Pf, kPiecesFp), lgPb = log2_pieces(Pb, kPiecesBp);
    if (lgPf < 0 || lgPb < 0 || max_items < 1) return cudaErrorInvalidValue;
    const size_t smem = sizeof(int) * ((size_t)max_items + 1);
    cudaError_t e = cudaSuccess;
    if (parts & kRoundFp)
        e = dispatch_t(xt, [&](auto *tx) {
            using T = std::remove_pointer_t<decltype(tx)>;
            auto go = [&](auto kern) {
                const unsigned blocks = persistent_blocks((const void *)kern, smem);
                kern<<<blocks, 256, smem, st>>>(scans, items, n_items, max_items, round, lgPf, sched);
            };
            if (lists) go(k_fp_batch<T, true>);
            else go(k_fp_batch<T, false>);
            return cudaGetLastError();
        });
    if (e != cudaSuccess) return e;
    if (parts & kRoundFused)
        e = dispatch_t(xt, [&](auto *tx) {
            using T = std::remove_pointer_t<decltype(tx)>;
            return dispatch_t(yt, [&](auto *ty) {
                using S = std::remove_pointer_t<decltype(ty)>;
                auto go = [&](auto kern) {
                    const unsigned blocks = persistent_blocks((const void *)kern, smem);
                    kern<<<blocks, 256, smem, st>>>(scans, items, n_items, max_items, round, lgPf, sched);
                };
                if (lists) go(k_sart_batch<T, S, true>);
                else go(k_sart_batch<T, S, false>);
                return cudaGetLastError();
            });
        });
    if (e != cudaSuccess) return e;
    if (parts & kRoundBp)
        e = dispatch_t(yt, [&](auto *ty) {
            using S = std::remove_pointer_t<decltype(ty)>;
            auto go = [&](auto kern) {
                const unsigned blocks = persistent_blocks((const void *)kern, smem, kBpBatchBlocksPerSm);
                kern<<<blocks, 256, smem, st>>>(scans, items, n_items, max_items, round, lgPb, sched);
            };
            if (lists) go(k_bp_batch<S, true>);
            else go(k_bp_batch<S, false>);
            return cudaGetLastError();
        });
    if (e != cudaSuccess || !(parts & kRoundUpdate)) return e;
    const dim3 grid_u((unsigned)std::min(update_blocks(max_vox), 512), max_items);
    return dispatch_t(x16t, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update_batch<X><<<grid_u, 256, 0, st>>>(scans, items, n_items, max_items, round);
        return cudaGetLastError();
    });
}

}  // namespace cylct
