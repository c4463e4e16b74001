// Device helpers of the ray-driven kernels: dtype conversion, predicated packed
// reductions, ray records and their equal-step pieces, and the self-resetting work
// counter of the persistent grids.
#pragma once

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

// Predicated packed reductions (the predicate is evaluated in PTX: no branch).
__device__ __forceinline__ void red_add2_if(bool c, float2 *p, float a, float b)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
                 "@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}"
                 ::"l"(p), "f"(a), "f"(b), "r"((unsigned)c) : "memory");
}

__device__ __forceinline__ void red_add4_if(bool c, float2 *p, float a, float b, float d, float e)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
                 "@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
                 ::"l"(p), "f"(a), "f"(b), "f"(d), "f"(e), "r"((unsigned)c) : "memory");
}

__device__ __forceinline__ void stage_trig_smem(const float2 *trig, int n_t, float2 *s)
{
    for (int k = threadIdx.x; k < n_t; k += blockDim.x) s[k] = trig[k];
    __syncthreads();
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

// --------------------------------------------------------------- SART update weights

// weight of voxel m (1 without a map); the element type is uniform over a launch
__device__ __forceinline__ float weight_at(const UpdateArgs &u, int64_t m)
{
    if (!u.w) return 1.f;
    switch (u.w_t) {
    case CYL_F16: return weight_f32(__ldg(static_cast<const __half *>(u.w) + m));
    case CYL_BF16: return weight_f32(__ldg(static_cast<const __nv_bfloat16 *>(u.w) + m));
    case CYL_U8: return weight_f32(__ldg(static_cast<const uint8_t *>(u.w) + m));
    default: return __ldg(static_cast<const float *>(u.w) + m);
    }
}

// weights of voxels 4i .. 4i + 3 in one aligned load (4, 8 or 16 bytes)
__device__ __forceinline__ float4 weight4_at(const UpdateArgs &u, int64_t i)
{
    if (!u.w) return make_float4(1.f, 1.f, 1.f, 1.f);
    switch (u.w_t) {
    case CYL_F16: {
        const uint2 r = __ldg(static_cast<const uint2 *>(u.w) + i);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    case CYL_BF16: {
        const uint2 r = __ldg(static_cast<const uint2 *>(u.w) + i);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    case CYL_U8: {
        const unsigned r = __ldg(static_cast<const unsigned *>(u.w) + i);
        return make_float4((float)(r & 0xffu), (float)((r >> 8) & 0xffu), (float)((r >> 16) & 0xffu),
                           (float)(r >> 24));
    }
    default: return __ldg(static_cast<const float4 *>(u.w) + i);
    }
}

// --------------------------------------------------------------- work scheduling

// sched[0] hands out warp tasks; sched[1] counts the warps that found no work left, and
// the last of them resets both, so the pair is zero again for the next launch on the
// stream.  Every warp of the grid calls retire() exactly once, after its last fetch has
// returned, so no fetch can follow the reset; no fence is needed (the kernel's end
// orders its memory operations before the next launch).
__device__ __forceinline__ int fetch_task(int *sched)
{
    int v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(sched, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ void retire(int *sched)
{
    if ((threadIdx.x & 31) == 0) {
        const unsigned total = gridDim.x * (blockDim.x >> 5);
        if ((unsigned)atomicAdd(sched + 1, 1) == total - 1) {
            atomicExch(sched, 0);
            atomicExch(sched + 1, 0);
        }
    }
}

// Warp task of fetch number f among n (f < task_span(n)): fetches f and f + 1 go to
// tasks about n / kStride apart.  Returns -1 for the few fetch numbers past n.
constexpr int kLgStride = 8, kStride = 1 << kLgStride;

__device__ __forceinline__ int64_t task_span(int64_t n) { return ((n + kStride - 1) >> kLgStride) << kLgStride; }

__device__ __forceinline__ int64_t task_of(int64_t f, int64_t n)
{
    const int64_t c = (n + kStride - 1) >> kLgStride;
    const int64_t t = (f & (kStride - 1)) * c + (f >> kLgStride);
    return t < n ? t : -1;
}

// Piece `piece` of P of ray rr: [ua, ub] from the recorded cuts (cut i of kSplit at
// u_in + frac_i (u_out - u_in)); false if empty.  Neighbouring pieces compute their
// shared cut from the same stored value, so the pieces tile the clipped interval.
__device__ __forceinline__ bool piece_bounds(const RayRec &rr, const uint16_t *__restrict__ cuts,
                                             int piece, int P, float &ua, float &ub)
{
    const float u0 = rr.c.x, u1 = rr.c.y;
    if (!(u1 > u0)) return false;
    const float len = u1 - u0;
    const int stride = kSplit / P;
    constexpr float kq = 1.f / 65535.f;
    ua = piece == 0 ? u0 : fminf(fmaf((float)__ldg(cuts + piece * stride - 1) * kq, len, u0), u1);
    ub = piece == P - 1 ? u1 : fminf(fmaf((float)__ldg(cuts + (piece + 1) * stride - 1) * kq, len, u0), u1);
    return ub > ua;
}

}  // namespace cylct
