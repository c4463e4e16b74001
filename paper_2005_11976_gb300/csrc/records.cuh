// Device helpers of the stored segment records (records.cu, gather.cu): the record
// format (FP32 length with the move to the next piece's voxel in its low 3 bits) and the
// predicated 4 x FP32 reduction of a voxel quad.
#pragma once

#include "device_common.cuh"

namespace cylct {

// voxel index change of each move code (codes whose changes coincide on a small grid are
// interchangeable: a replay only adds the change)
__host__ __device__ inline void move_deltas(int n_t, int n_r, int d[kRecMoves])
{
    const int st = n_r, sh = n_t * n_r, wrap = (n_t - 1) * n_r;
    d[0] = 1;       // shell +1
    d[1] = -1;      // shell -1
    d[2] = st;      // wedge +1
    d[3] = -st;     // wedge -1
    d[4] = -wrap;   // wedge N_theta - 1 -> 0
    d[5] = wrap;    // wedge 0 -> N_theta - 1
    d[6] = sh;      // slab +1
    d[7] = -sh;     // slab -1
}

__device__ __forceinline__ uint32_t move_code(int dd, const int d[kRecMoves])
{
    uint32_t c = kRecMoves - 1;
#pragma unroll
    for (int k = kRecMoves - 2; k >= 0; --k) c = dd == d[k] ? (uint32_t)k : c;
    return c;
}

__device__ __forceinline__ uint32_t rec_encode(float len, uint32_t code)
{
    return ((__float_as_uint(len) + 4u) & ~7u) | code;   // round to 20 mantissa bits
}

__device__ __forceinline__ float rec_len(uint32_t v) { return __uint_as_float(v & ~7u); }

__device__ __forceinline__ void red_add4f_if(bool c, float *p, float a, float b, float d, float e)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
                 "@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
                 ::"l"(p), "f"(a), "f"(b), "f"(d), "f"(e), "r"((unsigned)c) : "memory");
}

}  // namespace cylct
