// Per-ray and elementwise kernels of the SART path: ray records, row sums, weight
// scale, log transform, dtype conversion.  The traversal kernels are in rays.cu.
#include <type_traits>

#include "traverse.cuh"

namespace cylct {

size_t dtype_size(cyl_dtype t) { return t == CYL_F32 ? 4 : (t == CYL_U8 ? 1 : 2); }

template <class T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ------------------------------------------------------------------ ray records

__global__ void k_rays(GridDev g, const ProjGeom *__restrict__ geo, float4 *ra, float4 *rb, float4 *rc)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npix) return;
    const int p = blockIdx.y;
    RayRec rr = setup_ray(g, geo[p], (int)(j % g.det_w), (int)(j / g.det_w));
    const int64_t o = (int64_t)p * npix + j;
    ra[o] = rr.a;
    rb[o] = rr.b;
    rc[o] = rr.c;
}

// ------------------------------------------------------------------ row sums

__global__ void k_row_sums(ScanDev sd, int p0, float *L)
{
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npix) return;
    const float4 c = __ldg(sd.ray_c + (int64_t)(p0 + blockIdx.y) * npix + j);
    L[(int64_t)blockIdx.y * npix + j] = c.y > c.x ? c.z : 0.f;
}

// ------------------------------------------------------------ elementwise kernels

template <class W>
__global__ void k_wmax(const W *__restrict__ w, int64_t n, unsigned int *out)
{
    float v = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v = fmaxf(v, weight_f32(w[i]));
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
    const float l0 = logf(i0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float c = fmaxf(to_f32<I>(in[i]), 1.f);
        out[i] = from_f32<O>(l0 - logf(c));
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

static inline int elementwise_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_rays(const GridDev &g, const ProjGeom *geo, int n_proj, float4 *ra, float4 *rb,
                        float4 *rc, cudaStream_t st)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    k_rays<<<dim3((unsigned)((npix + 255) / 256), n_proj), 256, 0, st>>>(g, geo, ra, rb, rc);
    return cudaGetLastError();
}

// compact plans: L of the listed rays of views p0 .. p0+np-1 (the rest are 0)
__global__ void k_row_sums_list(ScanDev sd, RayList rl, int p0, int np, float *L)
{
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h, base = (int64_t)p0 * npix;
    const int64_t a0 = rl.act_off[p0], n = rl.act_off[p0 + np] - a0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 c = __ldg(sd.ray_c + a0 + i);
        L[(int64_t)rl.act[a0 + i] - base] = c.y > c.x ? c.z : 0.f;
    }
}

cudaError_t launch_row_sums(const ScanDev &sd, int p0, int np, float *L, cudaStream_t st, const RayList &rl)
{
    if (np <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    if (rl.act) {
        cudaError_t e = cudaMemsetAsync(L, 0, sizeof(float) * (size_t)np * npix, st);
        if (e != cudaSuccess) return e;
        k_row_sums_list<<<152 * 8, 256, 0, st>>>(sd, rl, p0, np, L);
        return cudaGetLastError();
    }
    k_row_sums<<<dim3((unsigned)((npix + 255) / 256), np), 256, 0, st>>>(sd, p0, L);
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

cudaError_t launch_weight_scale(const void *w, cyl_dtype w_t, int64_t n, int mode, float lambda, float *wscale,
                                cudaStream_t st)
{
    // wscale[0] receives lambda / max(w) (mode 1) or lambda (mode 0); wscale[1] is the
    // max-reduction word.
    unsigned int *bits = reinterpret_cast<unsigned int *>(wscale + 1);
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const unsigned nb = elementwise_blocks(n);
        switch (w_t) {
        case CYL_F32: k_wmax<<<nb, 256, 0, st>>>(static_cast<const float *>(w), n, bits); break;
        case CYL_F16: k_wmax<<<nb, 256, 0, st>>>(static_cast<const __half *>(w), n, bits); break;
        case CYL_BF16: k_wmax<<<nb, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(w), n, bits); break;
        case CYL_U8: k_wmax<<<nb, 256, 0, st>>>(static_cast<const uint8_t *>(w), n, bits); break;
        default: return cudaErrorInvalidValue;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_wscale<<<1, 1, 0, st>>>(bits, mode, lambda, wscale);
    return cudaGetLastError();
}

cudaError_t kernel_binary_version(int *v)
{
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k_wscale);
    if (e == cudaSuccess) *v = a.binaryVersion;
    return e;
}

}  // namespace cylct
