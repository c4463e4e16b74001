// Back-projection by gathering per voxel (Eq. 7 without atomics).  The stored segment
// records of a pose list, ray by ray, the voxel and length of every piece; their
// transpose lists, voxel by voxel and view by view, the (pixel, length) of every piece
// that crosses the voxel.  With it one thread per voxel forms
//     num_m = sum_j t_jm r_j,   den_m = sum_j t_jm   over the subset's rays,
// reading the subset's residuals (one float per ray, a few hundred KB that stay in L1
// and L2), and applies the update of Eq. 7 to x_m directly: the back-projection, the
// column sums and the update are one pass over the voxels, with no reduction into a
// shared accumulator.  The forward projection and the residuals come from the records'
// replay (k_rec_sart without its backward part).
//
// Transpose of view v (once per pose): count the pieces per voxel (integer reductions,
// replaying the records), scan the counts into offsets off[v][0 .. V] (a scan over tiles
// of 2048 counts, then over the tiles' sums), and replay the records again, each piece
// taking the next slot of its voxel (ent[ebase[v] + off[v][m] + ...] = (pixel, length)).
// The slots of a voxel are filled in no fixed order, so its sums' rounding may change
// from pose to pose; the values summed do not.
#include <algorithm>
#include <type_traits>

#include "records.cuh"

namespace cylct {

constexpr int kScanTile = 2048;   // counts per block of the tile scan (256 threads x 8)

// One warp per run of a task (the records' replay order), the 32 rays side by side.
// cnt != null: cnt[voxel] += 1 per piece.  Else each piece takes the next slot of its
// voxel from cur and writes (pixel, length) there in ent (the view's entries).
__global__ void __launch_bounds__(256) k_vox_pieces(RecDev rd, int64_t t0, int64_t n_task, uint32_t *cnt,
                                                    uint32_t *cur, uint2 *ent)
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
            if (cnt) {
#pragma unroll 4
                for (int64_t s = a; s < b; ++s) {
                    const uint32_t v = __ldg(rp + s * 32);
                    atomicAdd(cnt + idx, 1u);
                    idx += s_d[v & 7u];
                }
            } else {
                // four slots taken before the four entries are written, so that the
                // atomics' round trips overlap instead of each waiting on the last store
                for (int64_t s = a; s < b; s += 4) {
                    uint32_t v[4], slot[4];
                    int id[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = s + i < b ? __ldg(rp + (s + i) * 32) : 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        id[i] = idx;
                        idx += s_d[v[i] & 7u];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) slot[i] = s + i < b ? atomicAdd(cur + id[i], 1u) : 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (s + i < b) ent[slot[i]] = make_uint2((uint32_t)pix, v[i] & ~7u);
                }
            }
        }
        __syncwarp();
    }
}

// Exclusive scan of in[0 .. n) into out, tile by tile: each block scans kScanTile counts
// (8 consecutive per thread) and writes its tile's sum into tsum.
__global__ void __launch_bounds__(256) k_scan_tile(const uint32_t *__restrict__ in, uint32_t *out, int64_t n,
                                                   uint32_t *tsum)
{
    __shared__ uint32_t s_w[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 8;
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = base + i < n ? in[base + i] : 0u;
    uint32_t run = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t t = v[i];
        v[i] = run;
        run += t;
    }
    // exclusive scan of the threads' sums: within the warp, then across the 8 warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    uint32_t woff = 0, tot = 0;
    for (int q = 0; q < 8; ++q) {
        woff += q < wid ? s_w[q] : 0u;
        tot += s_w[q];
    }
    const uint32_t off = woff + incl - run;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (base + i < n) out[base + i] = v[i] + off;
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// Exclusive scan of the nt tile sums in place (one block of 1024 threads, a contiguous
// chunk each); *total receives their sum.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *tsum, int64_t nt, uint32_t *total)
{
    __shared__ uint32_t part[1024];
    const int64_t per = (nt + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(a + per, nt);
    uint32_t s = 0;
    for (int64_t i = a; i < b; ++i) s += tsum[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const uint32_t x = part[t];
            part[t] = run;
            run += x;
        }
        *total = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; ++i) {
        const uint32_t x = tsum[i];
        tsum[i] = run;
        run += x;
    }
}

// out[i] += the scanned sum of the tiles before i's
__global__ void k_scan_add(uint32_t *out, int64_t n, const uint32_t *__restrict__ tsum)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] += tsum[i / kScanTile];
}

// ebase[v + 1] = ebase[v] + the view's entry count (off[v][V])
__global__ void k_vox_base(int64_t *ebase, int v, const uint32_t *total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) ebase[v + 1] = ebase[v] + (int64_t)*total;
}

// sums of t r and t over the entries [e0, e1) of one voxel in one view: up to four entries
// and their residuals are loaded before any is used
__device__ __forceinline__ void vox_sums(const uint2 *__restrict__ ent, const float *__restrict__ rv, uint32_t e0,
                                         uint32_t e1, float &num, float &den)
{
    for (uint32_t e = e0; e < e1; e += 4) {
        uint2 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = e + k < e1 ? __ldg(ent + e + k) : make_uint2(0u, 0u);
        float r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = e + k < e1 ? __ldg(rv + q[k].x) : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float t = __uint_as_float(q[k].y);
            num = fmaf(t, r[k], num);
            den += t;
        }
    }
}

// Eq. 7 for the subset of views p0 .. p0+np-1, one voxel per thread (consecutive voxels in
// consecutive lanes, so that a warp's offsets, entries, x and w are contiguous): num and
// den gathered over the voxel's pieces in each view, then x_m += s w_m num_m /
// max(den_m, eps) where den_m > 0 (optionally x >= 0).  One view's den is summed in
// FP32 (a voxel meets about two pieces of a view, each length carrying 20 mantissa bits,
// so the sum is exact unless two of them differ by more than 16x); the views of a subset
// add in FP64.  resid holds the subset's residuals, view by view.
template <class X>
__global__ void __launch_bounds__(256) k_vox_sart(VoxDev vd, int p0, int np, const float *__restrict__ resid,
                                                  UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    X *x16 = static_cast<X *>(u.x16);
    const uint32_t nv = (uint32_t)vd.n_vox, stride = gridDim.x * blockDim.x;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < nv; m += stride) {
        float num = 0.f;
        double den = 0.0;
        for (int v = 0; v < np; ++v) {
            const uint32_t *off = vd.off + (int64_t)(p0 + v) * (vd.n_vox + 1);
            float dv = 0.f;
            vox_sums(vd.ent + __ldg(vd.ebase + p0 + v), resid + (int64_t)v * vd.npix, __ldg(off + m),
                     __ldg(off + m + 1), num, dv);
            den += (double)dv;
        }
        const float d = (float)den;
        if (d > 0.f) {
            float xv = u.strict16 ? as_f32<X>(x16[m]) : u.x32[m];
            xv = fmaf(sc * weight_at(u, m), num / fmaxf(d, vd.eps), xv);
            if (u.clamp) xv = fmaxf(xv, 0.f);
            if (!u.strict16) u.x32[m] = xv;
            if (x16) x16[m] = from_f32r<X>(xv);
        }
    }
}

// The same for a subset of one view (the kernel the default one-view subsets run),
// software-pipelined: while voxel m is summed, the offsets of voxel m + 2s (s: the grid's
// thread count) and the first kVoxQ entries, x and w of voxel m + s are already on their
// way, so a thread keeps three voxels' loads in flight instead of waiting on the offsets
// -> entries -> residuals chain of each.  The offsets and entries are read once per sweep
// and loaded evict-first, so that L2 keeps x, w and the residuals for the next subset's
// kernels.  The pieces are summed in entry order, as above (same rounding).
constexpr int kVoxQ = 4;

template <class X>
__global__ void __launch_bounds__(256, 6) k_vox_sart1(VoxDev vd, int p0, const float *__restrict__ resid,
                                                       UpdateArgs u)
{
    const float sc = u.wscale ? *u.wscale : u.lambda;
    X *x16 = static_cast<X *>(u.x16);
    const uint32_t *off = vd.off + (int64_t)p0 * (vd.n_vox + 1);
    const uint2 *ent = vd.ent + __ldg(vd.ebase + p0);
    const uint32_t nv = (uint32_t)vd.n_vox, stride = gridDim.x * blockDim.x;
    uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nv) return;   // no barrier below
    auto x_at = [&](uint32_t i) { return u.strict16 ? as_f32<X>(x16[i]) : u.x32[i]; };
    uint32_t a0 = __ldcs(off + m), a1 = __ldcs(off + m + 1), b0 = 0, b1 = 0;
    if (m + stride < nv) {
        b0 = __ldcs(off + m + stride);
        b1 = __ldcs(off + m + stride + 1);
    }
    uint2 q[kVoxQ];
#pragma unroll
    for (int k = 0; k < kVoxQ; ++k) q[k] = a0 + k < a1 ? __ldcs(ent + a0 + k) : make_uint2(0u, 0u);
    float xv = x_at(m), wv = weight_at(u, m);
    for (;;) {
        const uint32_t mn = m + stride, mnn = mn + stride;
        uint32_t c0 = 0, c1 = 0;
        if (mnn < nv) {
            c0 = __ldcs(off + mnn);
            c1 = __ldcs(off + mnn + 1);
        }
        uint2 qn[kVoxQ];
        float xn = 0.f, wn = 0.f;
#pragma unroll
        for (int k = 0; k < kVoxQ; ++k) qn[k] = make_uint2(0u, 0u);
        if (mn < nv) {
#pragma unroll
            for (int k = 0; k < kVoxQ; ++k)
                if (b0 + k < b1) qn[k] = __ldcs(ent + b0 + k);
            xn = x_at(mn);
            wn = weight_at(u, mn);
        }
        float r[kVoxQ];
#pragma unroll
        for (int k = 0; k < kVoxQ; ++k) r[k] = a0 + k < a1 ? __ldg(resid + q[k].x) : 0.f;
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k < kVoxQ; ++k) {
            const float t = __uint_as_float(q[k].y);   // 0 past the voxel's last piece
            num = fmaf(t, r[k], num);
            den += t;
        }
        if (a0 + kVoxQ < a1) vox_sums(ent, resid, a0 + kVoxQ, a1, num, den);
        if (den > 0.f) {
            xv = fmaf(sc * wv, num / fmaxf(den, vd.eps), xv);
            if (u.clamp) xv = fmaxf(xv, 0.f);
            if (!u.strict16) u.x32[m] = xv;
            if (x16) x16[m] = from_f32r<X>(xv);
        }
        if (mn >= nv) break;
        m = mn;
        a0 = b0;
        a1 = b1;
        b0 = c0;
        b1 = c1;
#pragma unroll
        for (int k = 0; k < kVoxQ; ++k) q[k] = qn[k];
        xv = xn;
        wv = wn;
    }
}

// ------------------------------------------------------------------ launchers

static unsigned item_blocks(const RecDev &rd, int64_t n_task)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(((n_task << rd.lgP) + 7) / 8, 152 * 8));
}

cudaError_t launch_vox_count(const RecDev &rd, int n_proj, int64_t n_vox, uint32_t *cnt, uint32_t *off,
                             uint32_t *tsum, int64_t *ebase, cudaStream_t st)
{
    const int64_t nt = (n_vox + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(ebase, 0, sizeof(int64_t), st);
    for (int v = 0; v < n_proj && e == cudaSuccess; ++v) {
        uint32_t *ov = off + (int64_t)v * (n_vox + 1);
        e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * n_vox, st);
        if (e != cudaSuccess) break;
        k_vox_pieces<<<item_blocks(rd, rd.tpv), 256, 0, st>>>(rd, (int64_t)v * rd.tpv, rd.tpv, cnt, nullptr, nullptr);
        k_scan_tile<<<(unsigned)nt, 256, 0, st>>>(cnt, ov, n_vox, tsum);
        k_scan_top<<<1, 1024, 0, st>>>(tsum, nt, ov + n_vox);
        k_scan_add<<<(unsigned)std::min<int64_t>((n_vox + 255) / 256, 152 * 8), 256, 0, st>>>(ov, n_vox, tsum);
        k_vox_base<<<1, 32, 0, st>>>(ebase, v, ov + n_vox);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_vox_fill(const RecDev &rd, int n_proj, int64_t n_vox, const uint32_t *off, const int64_t *h_ebase,
                            uint32_t *cur, uint2 *ent, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < n_proj && e == cudaSuccess; ++v) {
        e = cudaMemcpyAsync(cur, off + (int64_t)v * (n_vox + 1), sizeof(uint32_t) * n_vox, cudaMemcpyDeviceToDevice,
                            st);
        if (e != cudaSuccess) break;
        k_vox_pieces<<<item_blocks(rd, rd.tpv), 256, 0, st>>>(rd, (int64_t)v * rd.tpv, rd.tpv, nullptr, cur,
                                                              ent + h_ebase[v]);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_vox_sart(const VoxDev &vd, int p0, int np, const float *resid, const UpdateArgs &u,
                            cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((vd.n_vox + 255) / 256, 152 * 8));
    const cyl_dtype xt = u.x16 ? u.x16_t : CYL_F32;
    auto go = [&](auto *tx) {
        using X = std::remove_pointer_t<decltype(tx)>;
        if (np == 1)
            k_vox_sart1<X><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((vd.n_vox + 255) / 256, 152 * 6)),
                             256, 0, st>>>(vd, p0, resid, u);
        else k_vox_sart<X><<<blocks, 256, 0, st>>>(vd, p0, np, resid, u);
        return cudaGetLastError();
    };
    switch (xt) {
    case CYL_F16: return go((__half *)nullptr);
    case CYL_BF16: return go((__nv_bfloat16 *)nullptr);
    default: return go((float *)nullptr);
    }
}

}  // namespace cylct
