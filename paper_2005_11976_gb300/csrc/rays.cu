// Ray-driven kernels: each ray is cut into P pieces of equal length along the ray, and
// each piece is walked by one thread (a warp holds the same piece of 32 adjacent rays,
// so its lanes walk similar paths).
//   forward:  q_j += sum over the piece of t_jl x_l          (x gathered from L2 / HBM)
//   backward: nd_l += (t_jl y_j, t_jl)                        (one packed 2 x FP32 atomic
//             per piece of a ray in a voxel: numerator and column sum of Eq. 6 together)
//   update:   x_l += s w_l num_l / den_l where den_l > 0      (Eq. 6), elementwise
// The forward kernel also clears the spare accumulator (the one the previous subset's
// update has consumed), so no separate memset pass is needed.
#include <type_traits>

#include "traverse.cuh"

namespace cylct {

template <class T> __device__ __forceinline__ float as_f32(T v);
template <> __device__ __forceinline__ float as_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float as_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float as_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T> __device__ __forceinline__ T from_f32r(float v);
template <> __device__ __forceinline__ float from_f32r<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32r<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32r<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void red_add2(float2 *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

struct Piece {
    int64_t r;      // ray slot in [0, n_rays)
    int piece;
    bool valid;
};

__device__ __forceinline__ Piece piece_of(int64_t n_rays, int P, int64_t block0 = 0)
{
    Piece pc;
    const int64_t gw = ((block0 + blockIdx.x) * (int64_t)blockDim.x + threadIdx.x) >> 5;
    pc.piece = (int)(gw % P);
    pc.r = (gw / P) * 32 + (threadIdx.x & 31);
    pc.valid = pc.r < n_rays;
    return pc;
}

__device__ __forceinline__ Tile whole_grid(const GridDev &g)
{
    Tile t;
    t.t0 = 0;
    t.t1 = g.n_t;
    t.s0 = 0;
    t.s1 = g.n_h;
    t.full_circle = true;
    return t;
}

__device__ __forceinline__ void stage_trig_smem(const float2 *trig, int n_t, float2 *s)
{
    for (int k = threadIdx.x; k < n_t; k += blockDim.x) s[k] = trig[k];
    __syncthreads();
}

// piece [ua, ub] of ray rr; false if the ray misses the grid
__device__ __forceinline__ bool piece_interval(const RayRec &rr, int piece, int P, float &ua, float &ub)
{
    if (!(rr.c.y > rr.c.x)) return false;
    const float len = (rr.c.y - rr.c.x) / (float)P;
    ua = rr.c.x + piece * len;
    ub = piece == P - 1 ? rr.c.y : rr.c.x + (piece + 1) * len;
    return ub > ua;
}

__device__ __forceinline__ RayRec ray_at(const ScanDev &sd, int64_t rec)
{
    RayRec rr;
    rr.a = __ldg(sd.ray_a + rec);
    rr.b = __ldg(sd.ray_b + rec);
    rr.c = __ldg(sd.ray_c + rec);
    return rr;
}

__device__ __forceinline__ void zero_slice(float2 *buf, int64_t len, int64_t tid, int64_t nthreads)
{
    if (!buf) return;
    for (int64_t i = tid; i < len; i += nthreads) buf[i] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------------ device bodies

template <class T>
__device__ __forceinline__ void fp_piece(const ScanDev &sd, const float2 *s_trig, int p0, int64_t n_rays,
                                         int P, const T *__restrict__ x, float *__restrict__ q, Piece pc)
{
    if (!pc.valid) return;
    const GridDev &g = sd.g;
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const RayRec rr = ray_at(sd, (int64_t)p0 * npix + pc.r);
    float ua, ub;
    if (!piece_interval(rr, pc.piece, P, ua, ub)) return;
    const Tile t = whole_grid(g);
    Walker w;
    w.init(g, s_trig, t, rr, ua, ub);
    float acc = 0.f;
    auto op = [&](int idx, float len) { acc = fmaf(len, as_f32<T>(__ldg(x + idx)), acc); };
    while (w.step(g, s_trig, t, op)) {
    }
    if (acc != 0.f) atomicAdd(q + pc.r, acc);
}

template <class S, bool SART>
__device__ __forceinline__ void bp_piece(const ScanDev &sd, const float2 *s_trig, int p0, int64_t n_rays,
                                         int P, const S *__restrict__ y, const float *__restrict__ q,
                                         float2 *__restrict__ nd, float *__restrict__ num,
                                         float *__restrict__ den, Piece pc)
{
    if (!pc.valid) return;
    const GridDev &g = sd.g;
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const RayRec rr = ray_at(sd, (int64_t)p0 * npix + pc.r);
    float ua, ub;
    if (!piece_interval(rr, pc.piece, P, ua, ub)) return;
    float yv;
    if (SART) {
        const float L = rr.c.z;
        yv = L > 0.f ? (as_f32<S>(y[pc.r]) - q[pc.r]) / L : 0.f;
    } else {
        yv = as_f32<S>(y[pc.r]);
        if (yv == 0.f && !den) return;
    }
    const Tile t = whole_grid(g);
    Walker w;
    w.init(g, s_trig, t, rr, ua, ub);
    if (nd) {
        auto op = [&](int idx, float len) {
            if (len > 0.f) red_add2(nd + idx, len * yv, len);
        };
        while (w.step(g, s_trig, t, op)) {
        }
    } else {
        auto op = [&](int idx, float len) {
            if (len > 0.f) {
                atomicAdd(num + idx, len * yv);
                if (den) atomicAdd(den + idx, len);
            }
        };
        while (w.step(g, s_trig, t, op)) {
        }
    }
}

template <class X>
__device__ __forceinline__ void update_voxel(const UpdateArgs &u, int64_t m, float2 v, float sc)
{
    if (!(v.y > 0.f)) return;
    X *x16 = static_cast<X *>(u.x16);
    float xv = u.strict16 ? as_f32<X>(x16[m]) : u.x32[m];
    const float wm = u.w ? __ldg(u.w + m) : 1.f;
    xv = fmaf(sc * wm, v.x / v.y, xv);
    if (u.clamp) xv = fmaxf(xv, 0.f);
    if (!u.strict16) u.x32[m] = xv;
    if (x16) x16[m] = from_f32r<X>(xv);
}

// ------------------------------------------------------------------ single scan

template <class T, int P>
__global__ void __launch_bounds__(256)
k_fp_ray(ScanDev sd, int p0, int64_t n_rays, const T *__restrict__ x, float *__restrict__ q,
         float2 *zero_buf, int64_t zero_len)
{
    extern __shared__ float2 s_trig_ray[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig_ray);
    zero_slice(zero_buf, zero_len, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
    fp_piece<T>(sd, s_trig_ray, p0, n_rays, P, x, q, piece_of(n_rays, P));
}

template <class S, int P, bool SART>
__global__ void __launch_bounds__(256)
k_bp_ray(ScanDev sd, int p0, int64_t n_rays, const S *__restrict__ y, const float *__restrict__ q,
         float2 *nd, float *num, float *den)
{
    extern __shared__ float2 s_trig_ray[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig_ray);
    bp_piece<S, SART>(sd, s_trig_ray, p0, n_rays, P, y, q, nd, num, den, piece_of(n_rays, P));
}

template <class X>
__global__ void k_update_nd(int64_t n, const float2 *__restrict__ nd, UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x)
        update_voxel<X>(u, m, __ldg(nd + m), sc);
}

struct CountRayOp {
    unsigned int n;
};

template <int P>
__global__ void __launch_bounds__(256)
k_count_ray(ScanDev sd, int p0, int64_t n_rays, unsigned long long *counts)
{
    extern __shared__ float2 s_trig_ray[];
    stage_trig_smem(sd.trig, sd.g.n_t, s_trig_ray);
    const Piece pc = piece_of(n_rays, P);
    unsigned int n = 0;
    int view = 0;
    const GridDev &g = sd.g;
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    if (pc.valid) {
        view = (int)(pc.r / npix);
        const RayRec rr = ray_at(sd, (int64_t)p0 * npix + pc.r);
        float ua, ub;
        if (piece_interval(rr, pc.piece, P, ua, ub)) {
            const Tile t = whole_grid(g);
            Walker w;
            w.init(g, s_trig_ray, t, rr, ua, ub);
            auto op = [&](int, float len) { n += len > 0.f; };
            while (w.step(g, s_trig_ray, t, op)) {
            }
            // the cut at the start of a later piece splits one segment of the ray in two
            if (pc.piece > 0 && n > 0) --n;
        }
    }
    if (n) atomicAdd(counts + view, (unsigned long long)n);
}

// ------------------------------------------------------------------ batched rounds

// Blocks (x, item): item k of the round's items; x spans the item's ray pieces.  The
// forward kernel also clears the scan's spare accumulators (projections and nd) for the
// next round.
template <class T, int P>
__global__ void __launch_bounds__(256)
k_fp_ray_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
               const int *__restrict__ n_items, int max_items, int round)
{
    extern __shared__ float2 s_trig_ray[];
    const int k = blockIdx.y;
    if (k >= n_items[round]) return;
    const BatchItem it = items[(int64_t)round * max_items + k];
    const BatchScan &sc = scans[it.scan];
    stage_trig_smem(sc.sd.trig, sc.sd.g.n_t, s_trig_ray);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    zero_slice(sc.nd[it.buf ^ 1], sc.nd_len, tid, nth);
    for (int64_t i = tid; i < sc.q_len; i += nth) sc.q[it.buf ^ 1][i] = 0.f;
    const int64_t n_rays = (int64_t)it.np * sc.sd.g.det_w * sc.sd.g.det_h;
    fp_piece<T>(sc.sd, s_trig_ray, it.p0, n_rays, P, static_cast<const T *>(sc.x_proj), sc.q[it.buf],
                piece_of(n_rays, P));
}

template <class S, int P>
__global__ void __launch_bounds__(256)
k_bp_ray_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
               const int *__restrict__ n_items, int max_items, int round)
{
    extern __shared__ float2 s_trig_ray[];
    const int k = blockIdx.y;
    if (k >= n_items[round]) return;
    const BatchItem it = items[(int64_t)round * max_items + k];
    const BatchScan &sc = scans[it.scan];
    stage_trig_smem(sc.sd.trig, sc.sd.g.n_t, s_trig_ray);
    const int64_t npix = (int64_t)sc.sd.g.det_w * sc.sd.g.det_h;
    const int64_t n_rays = (int64_t)it.np * npix;
    const S *y = static_cast<const S *>(sc.sino) + (int64_t)it.p0 * npix;
    bp_piece<S, true>(sc.sd, s_trig_ray, it.p0, n_rays, P, y, sc.q[it.buf], sc.nd[it.buf], nullptr,
                      nullptr, piece_of(n_rays, P));
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

template <class F>
static cudaError_t dispatch_p(int P, F &&f)
{
    switch (P) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 4: return f(std::integral_constant<int, 4>());
    case 8: return f(std::integral_constant<int, 8>());
    }
    return cudaErrorInvalidValue;
}

static inline unsigned ray_blocks(int64_t n_rays, int P)
{
    const int64_t warps = ((n_rays + 31) / 32) * P;
    return (unsigned)((warps * 32 + 255) / 256);
}

static inline size_t trig_smem(int n_t) { return sizeof(float2) * (size_t)n_t; }

static inline int update_blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

cudaError_t launch_fp_rays(const ScanDev &sd, int P, int p0, int np, const void *x, cyl_dtype xt,
                           float *q, float2 *zero_buf, int64_t zero_len, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const int64_t n_rays = (int64_t)np * sd.g.det_w * sd.g.det_h;
    return dispatch_t(xt, [&](auto *tx) {
        using T = std::remove_pointer_t<decltype(tx)>;
        return dispatch_p(P, [&](auto pc) {
            k_fp_ray<T, decltype(pc)::value><<<ray_blocks(n_rays, pc), 256, trig_smem(sd.g.n_t), st>>>(
                sd, p0, n_rays, (const T *)x, q, zero_buf, zero_len);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_bp_rays(const ScanDev &sd, int P, int p0, int np, const void *y, cyl_dtype yt,
                           const float *q, float2 *nd, float *num, float *den, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const int64_t n_rays = (int64_t)np * sd.g.det_w * sd.g.det_h;
    return dispatch_t(yt, [&](auto *ty) {
        using S = std::remove_pointer_t<decltype(ty)>;
        return dispatch_p(P, [&](auto pc) {
            if (q)
                k_bp_ray<S, decltype(pc)::value, true><<<ray_blocks(n_rays, pc), 256, trig_smem(sd.g.n_t), st>>>(
                    sd, p0, n_rays, (const S *)y, q, nd, num, den);
            else
                k_bp_ray<S, decltype(pc)::value, false><<<ray_blocks(n_rays, pc), 256, trig_smem(sd.g.n_t), st>>>(
                    sd, p0, n_rays, (const S *)y, q, nd, num, den);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_update_nd(int64_t n_vox, const float2 *nd, const UpdateArgs &u, cudaStream_t st)
{
    const cyl_dtype xt = u.x16 ? u.x16_t : CYL_F32;
    return dispatch_t(xt, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update_nd<X><<<update_blocks(n_vox), 256, 0, st>>>(n_vox, nd, u);
        return cudaGetLastError();
    });
}

cudaError_t launch_count_rays(const ScanDev &sd, int p0, int np, unsigned long long *counts, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const int64_t n_rays = (int64_t)np * sd.g.det_w * sd.g.det_h;
    k_count_ray<4><<<ray_blocks(n_rays, 4), 256, trig_smem(sd.g.n_t), st>>>(sd, p0, n_rays, counts);
    return cudaGetLastError();
}

cudaError_t launch_batch_round_rays(const BatchScan *scans, const BatchItem *items, const int *n_items,
                                    int max_items, int round, int64_t max_rays, int64_t max_vox,
                                    int max_nt, int P, cyl_dtype xt, cyl_dtype yt, cyl_dtype x16t,
                                    cudaStream_t st)
{
    const dim3 grid_r(ray_blocks(max_rays, P), max_items);
    cudaError_t e = dispatch_t(xt, [&](auto *tx) {
        using T = std::remove_pointer_t<decltype(tx)>;
        return dispatch_p(P, [&](auto pc) {
            k_fp_ray_batch<T, decltype(pc)::value><<<grid_r, 256, trig_smem(max_nt), st>>>(
                scans, items, n_items, max_items, round);
            return cudaGetLastError();
        });
    });
    if (e != cudaSuccess) return e;
    e = dispatch_t(yt, [&](auto *ty) {
        using S = std::remove_pointer_t<decltype(ty)>;
        return dispatch_p(P, [&](auto pc) {
            k_bp_ray_batch<S, decltype(pc)::value><<<grid_r, 256, trig_smem(max_nt), st>>>(
                scans, items, n_items, max_items, round);
            return cudaGetLastError();
        });
    });
    if (e != cudaSuccess) return e;
    const dim3 grid_u((unsigned)std::min(update_blocks(max_vox), 512), max_items);
    return dispatch_t(x16t, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update_batch<X><<<grid_u, 256, 0, st>>>(scans, items, n_items, max_items, round);
        return cudaGetLastError();
    });
}

}  // namespace cylct
