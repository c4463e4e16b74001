// Kernels of the SART path: ray records, tiled forward projection, tiled matched
// back-projection with the fused SART update, row sums, segment counts, log transform,
// dtype conversion.
#include <type_traits>

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

__device__ __forceinline__ RayRec load_ray(const ScanDev &sd, int64_t r)
{
    RayRec rr;
    rr.a = __ldg(sd.ray_a + r);
    rr.b = __ldg(sd.ray_b + r);
    rr.c = __ldg(sd.ray_c + r);
    return rr;
}

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

// ----------------------------------------------------------- tile staging helpers

struct TileSpan {
    int tw, th, chunk, n;   // wedges, slabs, voxels per slab, voxels
};

__device__ __forceinline__ TileSpan span_of(const GridDev &g, const Tile &t)
{
    TileSpan s;
    s.tw = t.t1 - t.t0;
    s.th = t.s1 - t.s0;
    s.chunk = s.tw * g.n_r;
    s.n = s.th * s.chunk;
    return s;
}

// global voxel index of local voxel i of a tile
__device__ __forceinline__ int64_t tile_global(const GridDev &g, const Tile &t, const TileSpan &s, int i)
{
    const int lh = i / s.chunk, rem = i - lh * s.chunk;
    return ((int64_t)(t.s0 + lh) * g.n_t + t.t0) * g.n_r + rem;
}

__device__ __forceinline__ void stage_trig(const ScanDev &sd, float2 *s_trig)
{
    for (int k = threadIdx.x; k < sd.g.n_t; k += blockDim.x) s_trig[k] = sd.trig[k];
}

// ------------------------------------------------------------- forward projection

// per-block scratch of tile_walk_all: chunk counter and one 32-entry map per warp
struct WalkShared {
    int chunk;
    int map[kTileThreads / 32][32];
};

struct FpK {
    const float *x;      // the tile's voxels in shared memory
    float *q;            // the view's projections
    __device__ __forceinline__ float payload(int64_t, const RayRec &) const { return 0.f; }
    __device__ __forceinline__ void piece(int idx, float len, float &acc) const { acc = fmaf(len, x[idx], acc); }
    __device__ __forceinline__ void end(int64_t j, float acc) const
    {
        if (acc != 0.f) atomicAdd(q + j, acc);
    }
};

// One CTA per (tile, views): stage the tile's voxels in shared memory once, then walk
// every ray of views p0 .. p0+np-1 that crosses the tile, adding its partial line
// integral to q (q holds np views).
template <class T>
__device__ __forceinline__ void fp_tile_body(const ScanDev &sd, int tile, int p0, int np,
                                             const T *__restrict__ x, float *__restrict__ q,
                                             float4 *smem4, WalkShared &ws)
{
    const GridDev &g = sd.g;
    float2 *s_trig = reinterpret_cast<float2 *>(smem4);
    float *s_x = reinterpret_cast<float *>(s_trig + ((g.n_t + 1) & ~1));
    const Tile t = tile_of(sd.td, g, tile);
    const TileSpan s = span_of(g, t);
    stage_trig(sd, s_trig);
    for (int i = threadIdx.x; i < s.n; i += blockDim.x) s_x[i] = to_f32<T>(__ldg(x + tile_global(g, t, s, i)));
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    for (int v = 0; v < np; ++v) {
        const int p = p0 + v;
        const int4 bb = sd.bbox[(int64_t)p * sd.td.n_tiles + tile];
        if (threadIdx.x == 0) ws.chunk = 0;
        __syncthreads();
        if (!(bb.x > bb.z || bb.y > bb.w)) {
            const int64_t r0 = (int64_t)p * npix;
            FpK k{s_x, q + (int64_t)v * npix};
            tile_walk_all(g, s_trig, t, sd.ray_a + r0, sd.ray_b + r0, sd.ray_c + r0, bb, k,
                          &ws.chunk, ws.map[threadIdx.x >> 5]);
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kTileThreads)
k_fp_tile(ScanDev sd, int p0, const T *__restrict__ x, float *__restrict__ q)
{
    extern __shared__ float4 smem4[];
    __shared__ WalkShared ws;
    const int tile = blockIdx.x, v = blockIdx.y;
    const int4 bb = sd.bbox[(int64_t)(p0 + v) * sd.td.n_tiles + tile];
    if (bb.x > bb.z || bb.y > bb.w) return;
    fp_tile_body(sd, tile, p0 + v, 1, x, q + (int64_t)v * sd.g.det_w * sd.g.det_h, smem4, ws);
}

// ----------------------------------------------------------------- back-projection

// SART: payload = residual (p_j - q_j) / L_j; pure: payload = y_j.  Each piece adds
// len * payload to num and len to den in shared memory.
template <class S, bool SART, bool DEN>
struct BpK {
    float *num, *den;
    const S *y;          // the view's data
    const float *q;      // the view's forward projections (SART)
    __device__ __forceinline__ float payload(int64_t j, const RayRec &rr) const
    {
        if (SART) {
            const float L = rr.c.z;
            const float pj = to_f32<S>(y[j]), qj = q[j];
            return L > 0.f ? (pj - qj) / L : 0.f;
        }
        return to_f32<S>(y[j]);
    }
    __device__ __forceinline__ void piece(int idx, float len, float &yv) const
    {
        if (len > 0.f) {
            atomicAdd(num + idx, len * yv);
            if (DEN) atomicAdd(den + idx, len);
        }
    }
    __device__ __forceinline__ void end(int64_t, float) const {}
};

template <class X>
__device__ __forceinline__ void sart_update(const UpdateArgs &u, int64_t m, float num, float den, float sc)
{
    if (!(den > 0.f)) return;
    X *x16 = static_cast<X *>(u.x16);
    float xv = u.strict16 ? to_f32<X>(x16[m]) : u.x32[m];
    const float wm = u.w ? __ldg(u.w + m) : 1.f;
    xv = fmaf(sc * wm, num / den, xv);
    if (u.clamp) xv = fmaxf(xv, 0.f);
    if (!u.strict16) u.x32[m] = xv;
    if (x16) x16[m] = from_f32<X>(xv);
}

// One CTA per tile: accumulate num = A^T y and den = A^T 1 of the subset's views in
// shared memory (y = SART residual (p - q) / L, or the given data in pure mode), then
// either apply Eq. 6 to the tile's voxels (SART) or write num / den out (pure).
template <class S, class X, bool SART>
__device__ __forceinline__ void bp_tile_body(const ScanDev &sd, int tile, int p0, int np,
                                             const S *__restrict__ y, const float *__restrict__ q,
                                             const UpdateArgs &upd, float *__restrict__ num_out,
                                             float *__restrict__ den_out, float4 *smem4,
                                             WalkShared &ws)
{
    const GridDev &g = sd.g;
    float2 *s_trig = reinterpret_cast<float2 *>(smem4);
    const Tile t = tile_of(sd.td, g, tile);
    const TileSpan s = span_of(g, t);
    float *s_num = reinterpret_cast<float *>(s_trig + ((g.n_t + 1) & ~1));
    float *s_den = s_num + s.n;
    stage_trig(sd, s_trig);
    for (int i = threadIdx.x; i < s.n; i += blockDim.x) {
        s_num[i] = 0.f;
        s_den[i] = 0.f;
    }
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    for (int v = 0; v < np; ++v) {
        const int p = p0 + v;
        const int4 bb = sd.bbox[(int64_t)p * sd.td.n_tiles + tile];
        if (threadIdx.x == 0) ws.chunk = 0;
        __syncthreads();
        if (!(bb.x > bb.z || bb.y > bb.w)) {
            const int64_t r0 = (int64_t)p * npix, y0 = (int64_t)v * npix;
            if (SART || den_out) {
                BpK<S, SART, true> k{s_num, s_den, y + y0, SART ? q + y0 : nullptr};
                tile_walk_all(g, s_trig, t, sd.ray_a + r0, sd.ray_b + r0, sd.ray_c + r0, bb, k,
                              &ws.chunk, ws.map[threadIdx.x >> 5]);
            } else {
                BpK<S, SART, false> k{s_num, s_den, y + y0, nullptr};
                tile_walk_all(g, s_trig, t, sd.ray_a + r0, sd.ray_b + r0, sd.ray_c + r0, bb, k,
                              &ws.chunk, ws.map[threadIdx.x >> 5]);
            }
        }
        __syncthreads();
    }
    if (SART) {
        const float sc = upd.wscale ? *upd.wscale : upd.lambda;
        for (int i = threadIdx.x; i < s.n; i += blockDim.x)
            sart_update<X>(upd, tile_global(g, t, s, i), s_num[i], s_den[i], sc);
    } else {
        for (int i = threadIdx.x; i < s.n; i += blockDim.x) {
            const int64_t m = tile_global(g, t, s, i);
            num_out[m] = s_num[i];
            if (den_out) den_out[m] = s_den[i];
        }
    }
}

template <class S, class X, bool SART>
__global__ void __launch_bounds__(kTileThreads)
k_bp_tile(ScanDev sd, int p0, int np, const S *__restrict__ y, const float *__restrict__ q,
          UpdateArgs upd, float *__restrict__ num_out, float *__restrict__ den_out)
{
    extern __shared__ float4 smem4[];
    __shared__ WalkShared ws;
    bp_tile_body<S, X, SART>(sd, blockIdx.x, p0, np, y, q, upd, num_out, den_out, smem4, ws);
}

// ------------------------------------------------------------------ batched solve

// Round r of a batched solve works on items[r * max_items .. + n_items[r]): for each, one
// subset of one scan.  Blocks are (tile, item); tiles beyond a scan's tile count and
// items beyond the round's count exit at once.  The forward kernel also clears the
// scan's other projection buffer, which the next round accumulates into.
template <class T>
__global__ void __launch_bounds__(kTileThreads)
k_fp_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
           const int *__restrict__ n_items, int max_items, int round)
{
    extern __shared__ float4 smem4[];
    __shared__ WalkShared ws;
    const int k = blockIdx.y;
    if (k >= n_items[round]) return;
    const BatchItem it = items[(int64_t)round * max_items + k];
    const BatchScan &sc = scans[it.scan];
    const int tile = blockIdx.x;
    if (tile >= sc.sd.td.n_tiles) return;
    {   // clear the next round's buffer: tile t zeroes its share
        float *qc = sc.q[it.buf ^ 1];
        const int64_t n = sc.q_len;
        const int64_t a = n * tile / sc.sd.td.n_tiles, b = n * (tile + 1) / sc.sd.td.n_tiles;
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) qc[i] = 0.f;
    }
    fp_tile_body(sc.sd, tile, it.p0, it.np, static_cast<const T *>(sc.x_proj), sc.q[it.buf], smem4, ws);
}

template <class S, class X>
__global__ void __launch_bounds__(kTileThreads)
k_bp_batch(const BatchScan *__restrict__ scans, const BatchItem *__restrict__ items,
           const int *__restrict__ n_items, int max_items, int round)
{
    extern __shared__ float4 smem4[];
    __shared__ WalkShared ws;
    const int k = blockIdx.y;
    if (k >= n_items[round]) return;
    const BatchItem it = items[(int64_t)round * max_items + k];
    const BatchScan &sc = scans[it.scan];
    const int tile = blockIdx.x;
    if (tile >= sc.sd.td.n_tiles) return;
    const int64_t npix = (int64_t)sc.sd.g.det_w * sc.sd.g.det_h;
    const S *y = static_cast<const S *>(sc.sino) + (int64_t)it.p0 * npix;
    bp_tile_body<S, X, true>(sc.sd, tile, it.p0, it.np, y, sc.q[it.buf], sc.upd, nullptr, nullptr,
                             smem4, ws);
}

// ------------------------------------------------------------ counts, row sums

struct CountK {
    unsigned int *n;
    __device__ __forceinline__ float payload(int64_t, const RayRec &) const { return 0.f; }
    __device__ __forceinline__ void piece(int, float len, float &acc) const { acc += len > 0.f ? 1.f : 0.f; }
    __device__ __forceinline__ void end(int64_t, float acc) const { atomicAdd(n, (unsigned int)acc); }
};

__global__ void __launch_bounds__(kTileThreads)
k_count_tile(ScanDev sd, int p0, unsigned long long *counts)
{
    extern __shared__ float4 smem4[];
    __shared__ WalkShared ws;
    __shared__ unsigned int s_n;
    const GridDev &g = sd.g;
    const int tile = blockIdx.x, v = blockIdx.y, p = p0 + v;
    const int4 bb = sd.bbox[(int64_t)p * sd.td.n_tiles + tile];
    if (bb.x > bb.z || bb.y > bb.w) return;
    float2 *s_trig = reinterpret_cast<float2 *>(smem4);
    const Tile t = tile_of(sd.td, g, tile);
    stage_trig(sd, s_trig);
    if (threadIdx.x == 0) {
        ws.chunk = 0;
        s_n = 0;
    }
    __syncthreads();
    const int64_t r0 = (int64_t)p * g.det_w * g.det_h;
    CountK k{&s_n};
    tile_walk_all(g, s_trig, t, sd.ray_a + r0, sd.ray_b + r0, sd.ray_c + r0, bb, k, &ws.chunk,
                  ws.map[threadIdx.x >> 5]);
    __syncthreads();
    if (threadIdx.x == 0 && s_n) atomicAdd(counts + v, (unsigned long long)s_n);
}

__global__ void k_row_sums(ScanDev sd, int p0, float *L)
{
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npix) return;
    const float4 c = __ldg(sd.ray_c + (int64_t)(p0 + blockIdx.y) * npix + j);
    L[(int64_t)blockIdx.y * npix + j] = c.y > c.x ? c.z : 0.f;
}

// ------------------------------------------------------------ elementwise kernels

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

static inline size_t trig_bytes(const GridDev &g) { return sizeof(float2) * (size_t)((g.n_t + 1) & ~1); }

cudaError_t set_kernel_attributes()
{
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    auto set = [&](const void *fn) {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, fn);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     maxsm - (int)fa.sharedSizeBytes);
        if (r != cudaSuccess && e == cudaSuccess) e = r;
    };
    set((const void *)k_fp_tile<float>);
    set((const void *)k_fp_tile<__half>);
    set((const void *)k_fp_tile<__nv_bfloat16>);
#define CYL_SET_BP(S)                                                  \
    set((const void *)k_bp_tile<S, float, true>);                      \
    set((const void *)k_bp_tile<S, __half, true>);                     \
    set((const void *)k_bp_tile<S, __nv_bfloat16, true>);              \
    set((const void *)k_bp_tile<S, float, false>);
    CYL_SET_BP(float)
    CYL_SET_BP(__half)
    CYL_SET_BP(__nv_bfloat16)
#undef CYL_SET_BP
    set((const void *)k_count_tile);
    set((const void *)k_fp_batch<float>);
    set((const void *)k_fp_batch<__half>);
    set((const void *)k_fp_batch<__nv_bfloat16>);
#define CYL_SET_BB(S)                                  \
    set((const void *)k_bp_batch<S, float>);           \
    set((const void *)k_bp_batch<S, __half>);          \
    set((const void *)k_bp_batch<S, __nv_bfloat16>);
    CYL_SET_BB(float)
    CYL_SET_BB(__half)
    CYL_SET_BB(__nv_bfloat16)
#undef CYL_SET_BB
    return e;
}

cudaError_t launch_rays(const GridDev &g, const ProjGeom *geo, int n_proj, float4 *ra, float4 *rb,
                        float4 *rc, cudaStream_t st)
{
    const int64_t npix = (int64_t)g.det_w * g.det_h;
    k_rays<<<dim3((unsigned)((npix + 255) / 256), n_proj), 256, 0, st>>>(g, geo, ra, rb, rc);
    return cudaGetLastError();
}

cudaError_t launch_fp_tiles(const ScanDev &sd, int p0, int np, const void *vol, cyl_dtype vt,
                            float *q, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    return dispatch1(vt, [&](auto *tv) {
        using T = std::remove_pointer_t<decltype(tv)>;
        k_fp_tile<T><<<dim3(sd.td.n_tiles, np), kTileThreads, sd.td.smem_fp, st>>>(
            sd, p0, (const T *)vol, q);
        return cudaGetLastError();
    });
}

cudaError_t launch_bp_tiles(const ScanDev &sd, int p0, int np, const void *sino, cyl_dtype sdt,
                            const float *q, const UpdateArgs *upd, float *num_out, float *den_out,
                            cudaStream_t st)
{
    return dispatch1(sdt, [&](auto *ts) {
        using S = std::remove_pointer_t<decltype(ts)>;
        if (!upd) {
            UpdateArgs none{};
            k_bp_tile<S, float, false><<<sd.td.n_tiles, kTileThreads, sd.td.smem_bp, st>>>(
                sd, p0, np, (const S *)sino, q, none, num_out, den_out);
            return cudaGetLastError();
        }
        const cyl_dtype xt = upd->x16 ? upd->x16_t : CYL_F32;
        return dispatch1(xt, [&](auto *tx) {
            using X = std::remove_pointer_t<decltype(tx)>;
            k_bp_tile<S, X, true><<<sd.td.n_tiles, kTileThreads, sd.td.smem_bp, st>>>(
                sd, p0, np, (const S *)sino, q, *upd, nullptr, nullptr);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_batch_round(const BatchScan *scans, const BatchItem *items, const int *n_items,
                               int max_items, int round, int max_tiles, int smem_fp, int smem_bp,
                               cyl_dtype xt, cyl_dtype st_, cyl_dtype x16t, cudaStream_t st)
{
    const dim3 grid(max_tiles, max_items);
    cudaError_t e = dispatch1(xt, [&](auto *tx) {
        using T = std::remove_pointer_t<decltype(tx)>;
        k_fp_batch<T><<<grid, kTileThreads, smem_fp, st>>>(scans, items, n_items, max_items, round);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    return dispatch1(st_, [&](auto *ts) {
        using S = std::remove_pointer_t<decltype(ts)>;
        return dispatch1(x16t, [&](auto *tx) {
            using X = std::remove_pointer_t<decltype(tx)>;
            k_bp_batch<S, X><<<grid, kTileThreads, smem_bp, st>>>(scans, items, n_items, max_items, round);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_row_sums(const ScanDev &sd, int p0, int np, float *L, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)sd.g.det_w * sd.g.det_h;
    k_row_sums<<<dim3((unsigned)((npix + 255) / 256), np), 256, 0, st>>>(sd, p0, L);
    return cudaGetLastError();
}

cudaError_t launch_count(const ScanDev &sd, int p0, int np, unsigned long long *counts,
                         cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_count_tile<<<dim3(sd.td.n_tiles, np), kTileThreads, trig_bytes(sd.g), st>>>(sd, p0, counts);
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
    // wscale[0] receives lambda / max(w) (mode 1) or lambda (mode 0); wscale[1] is the
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
