// Kernels of the SART path: forward projection / residual, matched back-projection,
// SART update, row sums, segment counts, log transform, dtype conversion.
#include "traverse.cuh"

namespace cylct {

size_t dtype_size(cyl_dtype t) { return t == CYL_F32 ? 4 : 2; }

template <class T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <class T> __device__ __forceinline__ float ldg_f32(const T *p) { return to_f32<T>(__ldg(p)); }

// Map a thread to its ray: a warp covers a wu x (32/wu) pixel tile, a block 4 warps
// stacked along v; blockIdx.z is the projection within the subset.
struct RayIndex {
    int iu, iv;
    bool valid;
};

__device__ __forceinline__ RayIndex ray_of_thread(const GridDev &g, int wu)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wv = 32 / wu;
    RayIndex r;
    r.iu = blockIdx.x * wu + (lane % wu);
    r.iv = (blockIdx.y * 4 + warp) * wv + lane / wu;
    r.valid = r.iu < g.det_w && r.iv < g.det_h;
    return r;
}

__device__ __forceinline__ void load_trig(const float2 *trig, int n_t, float2 *sm)
{
    for (int k = threadIdx.x; k < n_t; k += blockDim.x) sm[k] = trig[k];
    __syncthreads();
}

template <class T>
struct GatherOp {
    const T *__restrict__ x;
    float acc;
    __device__ __forceinline__ void operator()(int idx, float seg) { acc = fmaf(seg, ldg_f32(x + idx), acc); }
};

// q = A x (cyl_project) when RESID is false; the SART residual (p - q) / L when true.
template <class T, class S, bool RESID>
__global__ void __launch_bounds__(128)
k_forward(GridDev g, const ProjGeom *__restrict__ geo, const float2 *__restrict__ trig, int p0,
          const T *__restrict__ x, const S *__restrict__ sino, int64_t sino_stride,
          void *__restrict__ out, int wu)
{
    extern __shared__ float2 s_trig[];
    load_trig(trig, g.n_t, s_trig);
    RayIndex ri = ray_of_thread(g, wu);
    if (!ri.valid) return;
    const int pl = blockIdx.z;
    const ProjGeom pg = geo[p0 + pl];
    Ray ry = setup_ray(g, pg, ri.iu, ri.iv);
    GatherOp<T> op{x, 0.f};
    if (ry.hit) walk_ray(g, s_trig, ry, op);
    const int64_t pix = (int64_t)ri.iv * g.det_w + ri.iu;
    const int64_t o = (int64_t)pl * g.det_w * g.det_h + pix;
    if (RESID) {
        float p = to_f32<S>(sino[(int64_t)pl * sino_stride + pix]);
        float r = (ry.hit && ry.L > 0.f) ? (p - op.acc) / ry.L : 0.f;
        static_cast<float *>(out)[o] = r;
    } else {
        static_cast<S *>(out)[o] = from_f32<S>(op.acc);
    }
}

struct ScatterOp {
    float *__restrict__ num;
    float *__restrict__ den;
    float y;
    __device__ __forceinline__ void operator()(int idx, float seg)
    {
        if (seg > 0.f) {
            atomicAdd(num + idx, seg * y);
            if (den) atomicAdd(den + idx, seg);
        }
    }
};

// num += A^T y, den += A^T 1 over the subset's rays (same walk as k_forward, so the
// transpose matches the projector piece by piece).
template <class Y>
__global__ void __launch_bounds__(128)
k_backproject(GridDev g, const ProjGeom *__restrict__ geo, const float2 *__restrict__ trig, int p0,
              const Y *__restrict__ y, float *__restrict__ num, float *__restrict__ den, int wu)
{
    extern __shared__ float2 s_trig[];
    load_trig(trig, g.n_t, s_trig);
    RayIndex ri = ray_of_thread(g, wu);
    if (!ri.valid) return;
    const int pl = blockIdx.z;
    const int64_t o = (int64_t)pl * g.det_w * g.det_h + (int64_t)ri.iv * g.det_w + ri.iu;
    float yv = to_f32<Y>(y[o]);
    if (yv == 0.f && den == nullptr) return;
    const ProjGeom pg = geo[p0 + pl];
    Ray ry = setup_ray(g, pg, ri.iu, ri.iv);
    if (!ry.hit) return;
    ScatterOp op{num, den, yv};
    walk_ray(g, s_trig, ry, op);
}

struct CountOp {
    unsigned int n;
    __device__ __forceinline__ void operator()(int, float seg) { n += seg > 0.f; }
};

__global__ void __launch_bounds__(128)
k_count(GridDev g, const ProjGeom *__restrict__ geo, const float2 *__restrict__ trig, int p0,
        unsigned long long *counts, int wu)
{
    extern __shared__ float2 s_trig[];
    load_trig(trig, g.n_t, s_trig);
    RayIndex ri = ray_of_thread(g, wu);
    CountOp op{0u};
    if (ri.valid) {
        Ray ry = setup_ray(g, geo[p0 + blockIdx.z], ri.iu, ri.iv);
        if (ry.hit) walk_ray(g, s_trig, ry, op);
    }
    unsigned int v = op.n;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(counts + blockIdx.z, (unsigned long long)v);
}

__global__ void k_row_sums(GridDev g, const ProjGeom *__restrict__ geo, int p0, float *L)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    const int iu = (int)(i % g.det_w), iv = (int)(i / g.det_w);
    Ray ry = setup_ray(g, geo[p0 + blockIdx.y], iu, iv);
    L[(int64_t)blockIdx.y * npix + i] = ry.hit ? ry.L : 0.f;
}

// x += wscale * w * num / den where den > 0 (Eq. 6), then clear num/den for the next
// subset.  X16 (if any) receives the rounded iterate; in strict mode it IS the iterate.
template <class X16>
__global__ void k_update(int64_t n, float *__restrict__ x32, X16 *__restrict__ x16, int strict16,
                         float *__restrict__ num, float *__restrict__ den,
                         const float *__restrict__ w, const float *__restrict__ wscale, float lambda,
                         int clamp)
{
    const float sc = wscale ? *wscale : lambda;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x) {
        float d = den[m];
        if (d > 0.f) {
            float wm = w ? __ldg(w + m) : 1.f;
            float xv = strict16 ? to_f32<X16>(x16[m]) : x32[m];
            xv = fmaf(sc * wm, num[m] / d, xv);
            if (clamp) xv = fmaxf(xv, 0.f);
            if (!strict16) x32[m] = xv;
            if (x16) x16[m] = from_f32<X16>(xv);
            num[m] = 0.f;
            den[m] = 0.f;
        }
    }
}

__global__ void k_wmax(const float *__restrict__ w, int64_t n, unsigned int *out)
{
    float v = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v = fmaxf(v, w[i]);
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(v));  // v >= 0: order-preserving
}

__global__ void k_wscale(const unsigned int *wmax_bits, int mode, float lambda, float *wscale)
{
    float m = __uint_as_float(*wmax_bits);
    *wscale = mode == 1 ? (m > 0.f ? lambda / m : 0.f) : lambda;
}

template <class I, class O>
__global__ void k_log(const I *__restrict__ in, float i0, O *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float c = fmaxf(to_f32<I>(in[i]), 1.f);
        out[i] = from_f32<O>(logf(i0) - logf(c));
    }
}

template <class I, class O>
__global__ void k_convert(const I *__restrict__ in, O *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = from_f32<O>(to_f32<I>(in[i]));
}

// ------------------------------------------------------------------ launchers

static inline dim3 ray_grid(const GridDev &g, int np, int wu)
{
    int wv = 32 / wu;
    return dim3((g.det_w + wu - 1) / wu, (g.det_h + 4 * wv - 1) / (4 * wv), np);
}

static inline size_t trig_smem(const GridDev &g) { return sizeof(float2) * (size_t)g.n_t; }

template <class F>
static cudaError_t dispatch1(cyl_dtype t, F &&f)
{
    switch (t) {
    case CYL_F32: return f((float *)nullptr);
    case CYL_F16: return f((__half *)nullptr);
    case CYL_BF16: return f((__nv_bfloat16 *)nullptr);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_project(const GridDev &g, const ProjGeom *geo, const float2 *trig, int p0,
                           int np, const void *vol, cyl_dtype vt, void *out, cyl_dtype ot,
                           TileShape ts, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    return dispatch1(vt, [&](auto *tv) {
        using T = std::remove_pointer_t<decltype(tv)>;
        return dispatch1(ot, [&](auto *to) {
            using S = std::remove_pointer_t<decltype(to)>;
            k_forward<T, S, false><<<ray_grid(g, np, ts.wu), ray_block(), trig_smem(g), st>>>(
                g, geo, trig, p0, (const T *)vol, (const S *)nullptr, 0, out, ts.wu);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_residual(const GridDev &g, const ProjGeom *geo, const float2 *trig, int p0,
                            int np, const void *vol, cyl_dtype vt, const void *sino,
                            cyl_dtype sdt, int64_t sino_proj_stride, float *res, TileShape ts,
                            cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    return dispatch1(vt, [&](auto *tv) {
        using T = std::remove_pointer_t<decltype(tv)>;
        return dispatch1(sdt, [&](auto *ts_) {
            using S = std::remove_pointer_t<decltype(ts_)>;
            k_forward<T, S, true><<<ray_grid(g, np, ts.wu), ray_block(), trig_smem(g), st>>>(
                g, geo, trig, p0, (const T *)vol, (const S *)sino, sino_proj_stride, res, ts.wu);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_backproject(const GridDev &g, const ProjGeom *geo, const float2 *trig, int p0,
                               int np, const void *y, cyl_dtype yt, float *num, float *den,
                               TileShape ts, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    return dispatch1(yt, [&](auto *ty) {
        using Y = std::remove_pointer_t<decltype(ty)>;
        k_backproject<Y><<<ray_grid(g, np, ts.wu), ray_block(), trig_smem(g), st>>>(
            g, geo, trig, p0, (const Y *)y, num, den, ts.wu);
        return cudaGetLastError();
    });
}

static inline int elementwise_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_update(int64_t n, float *x32, void *x16, cyl_dtype x16t, int strict16,
                          float *num, float *den, const float *w, const float *wscale,
                          float lambda, int clamp, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = elementwise_blocks(n);
    if (!x16) {
        k_update<float><<<nb, 256, 0, st>>>(n, x32, (float *)nullptr, 0, num, den, w, wscale,
                                            lambda, clamp);
        return cudaGetLastError();
    }
    return dispatch1(x16t, [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        k_update<X><<<nb, 256, 0, st>>>(n, x32, (X *)x16, strict16, num, den, w, wscale,
                                        lambda, clamp);
        return cudaGetLastError();
    });
}

cudaError_t launch_row_sums(const GridDev &g, const ProjGeom *geo, int p0, int np, float *L,
                            cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    int64_t npix = (int64_t)g.det_w * g.det_h;
    k_row_sums<<<dim3((unsigned)((npix + 255) / 256), np), 256, 0, st>>>(g, geo, p0, L);
    return cudaGetLastError();
}

cudaError_t launch_count(const GridDev &g, const ProjGeom *geo, const float2 *trig, int p0,
                         int np, unsigned long long *counts, TileShape ts, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_count<<<ray_grid(g, np, ts.wu), ray_block(), trig_smem(g), st>>>(g, geo, trig, p0, counts,
                                                                        ts.wu);
    return cudaGetLastError();
}

cudaError_t launch_log(const void *in, cyl_dtype it, double i0, void *out, cyl_dtype ot,
                       int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    return dispatch1(it, [&](auto *ti) {
        using I = std::remove_pointer_t<decltype(ti)>;
        return dispatch1(ot, [&](auto *to) {
            using O = std::remove_pointer_t<decltype(to)>;
            k_log<I, O><<<elementwise_blocks(n), 256, 0, st>>>((const I *)in, (float)i0, (O *)out, n);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_convert(const void *in, cyl_dtype it, void *out, cyl_dtype ot, int64_t n,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    return dispatch1(it, [&](auto *ti) {
        using I = std::remove_pointer_t<decltype(ti)>;
        return dispatch1(ot, [&](auto *to) {
            using O = std::remove_pointer_t<decltype(to)>;
            k_convert<I, O><<<elementwise_blocks(n), 256, 0, st>>>((const I *)in, (O *)out, n);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_weight_scale(const float *w, int64_t n, int mode, float lambda, float *wscale,
                                cudaStream_t st)
{
    // wscale[0] holds lambda / max(w) (mode 1) or lambda (mode 0); wscale[1] is the
    // max-reduction word.
    unsigned int *bits = reinterpret_cast<unsigned int *>(wscale + 1);
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_wmax<<<elementwise_blocks(n), 256, 0, st>>>(w, n, bits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_wscale<<<1, 1, 0, st>>>(bits, mode, lambda, wscale);
    return cudaGetLastError();
}

}  // namespace cylct
