// Projection-based pose estimation (Sec. 2.1, Eq. 3-4) and the azimuthal phase of the
// part (Sec. 2.1, Eq. 5).
//
// k_corners    threshold + dilation + corner pixels of every projection, in one pass
//              over the detector rows (HBM-bound: every pixel is read once).
// k_track      Levenberg-Marquardt for the axis points (one warp per point, FP64), and
//              the pose from the two points.
// k_band       grey-value moments of the band along the projected axis.
// k_theta_mean the azimuthal mean of a volume; k_phase the first-harmonic fits.
//
// Corner keys.  Dilating the thresholded set M by the square S (clipped to the window W)
// gives D = (M + S) n W; the pixel of D that maximises a diagonal key (for example
// iu + iv, ties to the larger iv) is the best over m in M of the best pixel of the clipped
// square around m, and that pixel is the square's corner in the key's direction.  So the
// kernel never forms D: each thresholded pixel offers its clipped square's corner, and
// within a row only the leftmost and rightmost thresholded pixels can win.  A key packs
// the diagonal value (offset to stay positive) above the tie-break coordinate, so one
// 64-bit max over all candidates gives the corner exactly.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "plan.h"

namespace cylct {
namespace {

constexpr long long kKeyOff = 1ll << 20;   // |diagonal value| < 2^19 for sides <= 2^18 - 1
constexpr int kCornerThreads = 256;
constexpr int kOutPose = 20;               // doubles per scan of k_track's pose output
constexpr double kPi = 3.14159265358979323846;

// One scan of a corner launch: rows [row0, row0 + n_proj (v1 - v0)) of the launch.
struct CornerScan {
    const void *sino;
    int64_t row0;
    int64_t view0;            // index of the scan's first projection in keys / counts
    int n_proj, W, H;
    int u0, u1, v0, v1;
    int k;
    int vec;                  // rows start on 16-byte boundaries
    float thr;                // largest float <= threshold
};

// Per-projection geometry of the point tracking, stage coordinates (FP64).
struct ViewLM {
    double S[3], D0[3], du[3], dv[3];
    double e1[3], e2[3], n[3];   // dual basis of (du, dv) in the detector plane, normal
    double a0, b0, c0;           // e1 . (S - D0), e2 . (S - D0), n . (D0 - S)
    double su, sv;               // |du|, |dv|
};

struct TrackScan {
    int64_t view0;
    int n_proj, H, max_iter;
    double gamma;
};

// Band constants of one projection (FP32, see cyl_band_moments).
struct BandView {
    float Au, Av, cdu, cdv, csu, csv;
};

__host__ __device__ inline void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__host__ __device__ inline double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------------------ corners

__device__ __forceinline__ unsigned long long corner_key(long long diag, int sec)
{
    return ((unsigned long long)(diag + kKeyOff) << 32) | (unsigned)sec;
}

// Keys of TL, TR, BL, BR offered by the thresholded pixels umin .. umax of row v.
__device__ __forceinline__ void offer_row(const CornerScan &cs, int v, int umin, int umax,
                                          unsigned long long key[4])
{
    const int ul = max(umin - cs.k, cs.u0), ur = min(umax + cs.k, cs.u1 - 1);
    const int vt = min(v + cs.k, cs.v1 - 1), vb = max(v - cs.k, cs.v0);
    key[0] = max(key[0], corner_key((long long)vt - ul, vt));
    key[1] = max(key[1], corner_key((long long)ur + vt, vt));
    key[2] = max(key[2], corner_key(-(long long)ul - vb, cs.H - 1 - vb));
    key[3] = max(key[3], corner_key((long long)ur - vb, cs.H - 1 - vb));
}

__device__ __forceinline__ void flush_corners(int64_t view, unsigned long long key[4],
                                              unsigned long long cnt, unsigned long long *keys,
                                              unsigned long long *counts)
{
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) key[c] = max(key[c], __shfl_xor_sync(0xffffffffu, key[c], o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && view >= 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (key[c]) atomicMax(keys + 4 * view + c, key[c]);
        if (cnt) atomicAdd(counts + view, cnt);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) key[c] = 0;
}

template <class T>
__device__ __forceinline__ void scan_elem(T x, int col, const CornerScan &cs, int &umin, int &umax,
                                          unsigned long long &cnt)
{
    const bool fg = col >= cs.u0 && col < cs.u1 && as_f32(x) > cs.thr;
    umin = fg ? min(umin, col) : umin;
    umax = fg ? max(umax, col) : umax;
    cnt += fg;
}

// Largest element of a 16-byte vector, as a float (NaN elements are passed over: a NaN
// never exceeds the threshold, and neither does the max of the others because of it).
__device__ __forceinline__ float vec_max(const uint4 &q, float)
{
    return fmaxf(fmaxf(__uint_as_float(q.x), __uint_as_float(q.y)),
                 fmaxf(__uint_as_float(q.z), __uint_as_float(q.w)));
}

__device__ __forceinline__ float vec_max(const uint4 &q, __half)
{
    const __half2 *h = reinterpret_cast<const __half2 *>(&q);
    const __half2 m = __hmax2(__hmax2(h[0], h[1]), __hmax2(h[2], h[3]));
    return fmaxf(__low2float(m), __high2float(m));
}

__device__ __forceinline__ float vec_max(const uint4 &q, __nv_bfloat16)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
    const __nv_bfloat162 m = __hmax2(__hmax2(h[0], h[1]), __hmax2(h[2], h[3]));
    return fmaxf(__low2float(m), __high2float(m));
}

// One warp per chunk of `rows_per_warp` consecutive rows of the launch; lanes split each
// row's columns (16-byte loads where the rows are aligned).
template <class T>
__global__ void __launch_bounds__(kCornerThreads)
k_corners(const CornerScan *__restrict__ scans, int n_scans, int64_t rows_total,
          int64_t rows_per_warp, unsigned long long *keys, unsigned long long *counts)
{
    constexpr int V = 16 / sizeof(T);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t r0 = warp * rows_per_warp;
    const int64_t r1 = min(r0 + rows_per_warp, rows_total);
    if (r0 >= r1) return;
    int s = 0;
    {   // last scan whose first row is <= r0
        int lo = 0, hi = n_scans - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (scans[mid].row0 <= r0) lo = mid;
            else hi = mid - 1;
        }
        s = lo;
    }
    CornerScan cs = scans[s];
    int64_t view = -1;
    unsigned long long key[4] = {0, 0, 0, 0}, cnt = 0;
    for (int64_t r = r0; r < r1; ++r) {
        while (s + 1 < n_scans && r >= scans[s + 1].row0) cs = scans[++s];
        const int64_t local = r - cs.row0;
        const int rows = cs.v1 - cs.v0;
        const int p = (int)(local / rows);
        const int v = cs.v0 + (int)(local - (int64_t)p * rows);
        if (cs.view0 + p != view) {
            flush_corners(view, key, cnt, keys, counts);
            cnt = 0;
            view = cs.view0 + p;
        }
        const T *row = static_cast<const T *>(cs.sino) + ((int64_t)p * cs.H + v) * cs.W;
        int umin = INT_MAX, umax = -1;
        if (cs.vec) {
            // all of a row's loads are issued before any is used (U per lane in flight);
            // a vector with no element above the threshold is skipped after one packed max
            constexpr int U = 8;
            const int c0 = cs.u0 & ~(V - 1);
            for (int cb = c0 + lane * V; cb < cs.u1; cb += 32 * V * U) {
                uint4 q[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int c = cb + j * 32 * V;
                    q[j] = c < cs.u1 ? __ldg(reinterpret_cast<const uint4 *>(row + c)) : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int c = cb + j * 32 * V;
                    if (c < cs.u1 && vec_max(q[j], T()) > cs.thr) {
                        const T *e = reinterpret_cast<const T *>(&q[j]);
#pragma unroll
                        for (int i = 0; i < V; ++i) scan_elem(e[i], c + i, cs, umin, umax, cnt);
                    }
                }
            }
        } else {
            for (int c = cs.u0 + lane; c < cs.u1; c += 32) scan_elem(__ldg(row + c), c, cs, umin, umax, cnt);
        }
        if (umax >= 0) offer_row(cs, v, umin, umax, key);
    }
    flush_corners(view, key, cnt, keys, counts);
}

// Pixel (iu, iv) of corner c from its key (key != 0).
__host__ __device__ inline void decode_corner(unsigned long long key, int c, int H, int &iu, int &iv)
{
    const long long diag = (long long)(key >> 32) - kKeyOff;
    const int sec = (int)(key & 0xffffffffu);
    iv = c < 2 ? sec : H - 1 - sec;
    switch (c) {
    case 0: iu = (int)(iv - diag); break;    // -iu + iv
    case 1: iu = (int)(diag - iv); break;    //  iu + iv
    case 2: iu = (int)(-diag - iv); break;   // -iu - iv
    default: iu = (int)(diag + iv); break;   //  iu - iv
    }
}

__global__ void k_decode_corners(const unsigned long long *keys, int n_proj, int H, int32_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * n_proj) return;
    int iu = -1, iv = -1;
    if (keys[i]) decode_corner(keys[i], i & 3, H, iu, iv);
    out[2 * i] = iu;
    out[2 * i + 1] = iv;
}

// ------------------------------------------------------------------ point tracking

// Observed detector coordinates of one track in projection i: from the corner keys (mode
// 0: top pair, 1: bottom pair) or from an explicit track (mode 2; NaN = not observed).
struct Obs {
    const unsigned long long *keys;
    const double *track;
    int mode, H;
    __device__ bool at(int64_t i, double &a, double &b) const
    {
        if (mode == 2) {
            a = track[2 * i];
            b = track[2 * i + 1];
            return !(isnan(a) || isnan(b));
        }
        const unsigned long long k0 = keys[4 * i + 2 * mode], k1 = keys[4 * i + 2 * mode + 1];
        if (!k0 || !k1) return false;
        int u0, v0, u1, v1;
        decode_corner(k0, 2 * mode, H, u0, v0);
        decode_corner(k1, 2 * mode + 1, H, u1, v1);
        a = 0.5 * (double)(u0 + u1);
        b = 0.5 * (double)(v0 + v1);
        return true;
    }
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Residuals r = (obs - V(X)) scaled to mm, and J = dV/dX scaled alike, summed into the
// normal equations over the lane's projections, then over the warp (all lanes end with
// the same sums: A (6 upper entries), g = J^T r (3), cost).
__device__ void normal_eqs(const ViewLM *__restrict__ vw, int64_t view0, int n, const Obs &obs,
                           const double X[3], double acc[10])
{
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) {
        double ao, bo;
        if (!obs.at(view0 + i, ao, bo)) continue;
        const ViewLM &v = vw[view0 + i];
        const double Y[3] = {X[0] - v.S[0], X[1] - v.S[1], X[2] - v.S[2]};
        const double nY = dot3(v.n, Y), e1Y = dot3(v.e1, Y), e2Y = dot3(v.e2, Y);
        const double t = v.c0 / nY;
        const double r0 = (ao - (v.a0 + t * e1Y)) * v.su;
        const double r1 = (bo - (v.b0 + t * e2Y)) * v.sv;
        double J0[3], J1[3];
        for (int k = 0; k < 3; ++k) {
            J0[k] = t * (v.e1[k] - v.n[k] * e1Y / nY) * v.su;
            J1[k] = t * (v.e2[k] - v.n[k] * e2Y / nY) * v.sv;
        }
        acc[0] += J0[0] * J0[0] + J1[0] * J1[0];
        acc[1] += J0[0] * J0[1] + J1[0] * J1[1];
        acc[2] += J0[0] * J0[2] + J1[0] * J1[2];
        acc[3] += J0[1] * J0[1] + J1[1] * J1[1];
        acc[4] += J0[1] * J0[2] + J1[1] * J1[2];
        acc[5] += J0[2] * J0[2] + J1[2] * J1[2];
        acc[6] += J0[0] * r0 + J1[0] * r1;
        acc[7] += J0[1] * r0 + J1[1] * r1;
        acc[8] += J0[2] * r0 + J1[2] * r1;
        acc[9] += r0 * r0 + r1 * r1;
    }
    for (int q = 0; q < 10; ++q) acc[q] = warp_sum(acc[q]);
}

// Solves M d = g for the symmetric 3x3 M given by its upper entries (Cramer's rule);
// false when M is singular or the result is not finite.
__device__ bool solve3(const double m[6], const double g[3], double d[3])
{
    const double a = m[0], b = m[1], c = m[2], e = m[3], f = m[4], i = m[5];
    const double c00 = e * i - f * f, c01 = c * f - b * i, c02 = b * f - c * e;
    const double det = a * c00 + b * c01 + c * c02;
    if (det == 0.0 || !isfinite(det)) return false;
    const double c11 = a * i - c * c, c12 = b * c - a * f, c22 = a * e - b * b;
    d[0] = (c00 * g[0] + c01 * g[1] + c02 * g[2]) / det;
    d[1] = (c01 * g[0] + c11 * g[1] + c12 * g[2]) / det;
    d[2] = (c02 * g[0] + c12 * g[1] + c22 * g[2]) / det;
    return isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]);
}

// Eq. 4 by Levenberg-Marquardt for one track; every lane of the warp ends with the same
// result.  Returns the number of observed projections.
__device__ int track_lm(const ViewLM *__restrict__ vw, int64_t view0, int n, const Obs &obs,
                        int max_iter, double X[3], double &rms, int &iters)
{
    int first = INT_MAX, nobs = 0;
    for (int i = threadIdx.x & 31; i < n; i += 32) {
        double a, b;
        if (obs.at(view0 + i, a, b)) {
            first = min(first, i);
            ++nobs;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        nobs += __shfl_xor_sync(0xffffffffu, nobs, o);
    }
    iters = 0;
    if (nobs < 2) {
        X[0] = X[1] = X[2] = rms = nan("");
        return nobs;
    }
    {   // start on the first observed projection's ray, at the stage origin's distance
        double a, b;
        obs.at(view0 + first, a, b);
        const ViewLM &v = vw[view0 + first];
        double P[3], len = 0.0;
        for (int k = 0; k < 3; ++k) {
            P[k] = v.D0[k] + a * v.du[k] + b * v.dv[k] - v.S[k];
            len += P[k] * P[k];
        }
        const double f = sqrt(dot3(v.S, v.S)) / sqrt(len);
        for (int k = 0; k < 3; ++k) X[k] = v.S[k] + f * P[k];
    }
    double mu = 1e-3, acc[10];
    normal_eqs(vw, view0, n, obs, X, acc);
    double cost = acc[9];
    while (iters < max_iter) {
        ++iters;
        const double m[6] = {acc[0] * (1.0 + mu), acc[1], acc[2], acc[3] * (1.0 + mu), acc[4],
                             acc[5] * (1.0 + mu)};
        double d[3];
        if (!solve3(m, acc + 6, d)) {
            mu *= 10.0;
            if (mu > 1e15) break;
            continue;
        }
        const double Xn[3] = {X[0] + d[0], X[1] + d[1], X[2] + d[2]};
        double accn[10];
        normal_eqs(vw, view0, n, obs, Xn, accn);     // the trial's cost and, if kept, its equations
        const bool keep = accn[9] < cost;
        const double *Xr = keep ? Xn : X;
        const bool small = sqrt(dot3(d, d)) <= 1e-10 * (1.0 + sqrt(dot3(Xr, Xr)));
        if (keep) {
            X[0] = Xn[0];
            X[1] = Xn[1];
            X[2] = Xn[2];
            mu = fmax(mu / 10.0, 1e-15);
            for (int q = 0; q < 10; ++q) acc[q] = accn[q];
            cost = acc[9];
        } else {
            mu *= 10.0;
        }
        if (small || mu > 1e15) break;
    }
    rms = sqrt(cost / nobs);
    return nobs;
}

// Pose mode (tracks from keys): block of 64 threads per scan, warp 0 the top track, warp 1
// the bottom track; out[scan][kOutPose] = top xyz, bottom xyz, rms top, rms bottom,
// steps top, steps bottom, n_views, status, alpha, beta, gamma, tx, ty, tz.
__global__ void __launch_bounds__(64)
k_track_pose(const TrackScan *__restrict__ scans, const ViewLM *__restrict__ vw,
             const unsigned long long *__restrict__ keys, double *out)
{
    __shared__ double sh[2][5];
    __shared__ int nv[2];
    const TrackScan ts = scans[blockIdx.x];
    const int w = threadIdx.x >> 5;
    Obs obs{keys, nullptr, w, ts.H};
    double X[3], rms;
    int iters;
    const int nobs = track_lm(vw, ts.view0, ts.n_proj, obs, ts.max_iter, X, rms, iters);
    if ((threadIdx.x & 31) == 0) {
        sh[w][0] = X[0];
        sh[w][1] = X[1];
        sh[w][2] = X[2];
        sh[w][3] = rms;
        sh[w][4] = iters;
        nv[w] = nobs;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double *o = out + (int64_t)blockIdx.x * kOutPose;
    for (int k = 0; k < 3; ++k) {
        o[k] = sh[0][k];
        o[3 + k] = sh[1][k];
    }
    o[6] = sh[0][3];
    o[7] = sh[1][3];
    o[8] = sh[0][4];
    o[9] = sh[1][4];
    o[10] = nv[0];
    const bool ok = nv[0] >= 2;   // both tracks come from the same projections
    o[11] = ok ? 0.0 : 1.0;
    double pose[6] = {0.0, 0.0, ts.gamma, 0.0, 0.0, 0.0};
    if (ok) {
        double ax[3], len = 0.0;
        for (int k = 0; k < 3; ++k) {
            ax[k] = sh[0][k] - sh[1][k];
            len += ax[k] * ax[k];
        }
        len = sqrt(len);
        for (int k = 0; k < 3; ++k) ax[k] /= len;
        pose[1] = acos(fmin(1.0, fmax(-1.0, ax[2])));
        pose[0] = hypot(ax[0], ax[1]) > 1e-15 ? atan2(ax[0], -ax[1]) : 0.0;
        for (int k = 0; k < 3; ++k) pose[3 + k] = 0.5 * (sh[0][k] + sh[1][k]);
    }
    for (int k = 0; k < 6; ++k) o[12 + k] = pose[k];
}

// Track mode: one warp; out = x, y, z, rms, steps.
__global__ void __launch_bounds__(32)
k_track_one(const ViewLM *__restrict__ vw, int n, const double *__restrict__ track, int max_iter,
            double *out)
{
    Obs obs{nullptr, track, 2, 0};
    double X[3], rms;
    int iters;
    track_lm(vw, 0, n, obs, max_iter, X, rms, iters);
    if (threadIdx.x == 0) {
        out[0] = X[0];
        out[1] = X[1];
        out[2] = X[2];
        out[3] = rms;
        out[4] = iters;
    }
}

// ------------------------------------------------------------------ band moments

// One warp per chunk of rows of one sinogram; FP32 band test (no contraction), FP64 sums.
template <class T>
__global__ void __launch_bounds__(kCornerThreads)
k_band(const T *__restrict__ sino, int n_proj, int W, int H, const BandView *__restrict__ bv,
       float half_width, int64_t rows_per_warp, double *moments)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t rows_total = (int64_t)n_proj * H;
    const int64_t r0 = warp * rows_per_warp;
    const int64_t r1 = min(r0 + rows_per_warp, rows_total);
    int p = -1;
    BandView b{};
    double m0 = 0.0, m1 = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const int pr = (int)(r / H);
        if (pr != p) {
            if (p >= 0) {
                m0 = warp_sum(m0);
                m1 = warp_sum(m1);
                if (lane == 0) {
                    atomicAdd(moments + 2 * p, m0);
                    atomicAdd(moments + 2 * p + 1, m1);
                }
                m0 = m1 = 0.0;
            }
            p = pr;
            b = bv[p];
        }
        const int v = (int)(r - (int64_t)pr * H);
        const float fb = __fsub_rn((float)v, b.Av);
        const float db = __fmul_rn(fb, b.cdv), sb = __fmul_rn(fb, b.csv);
        const T *row = sino + r * W;
        for (int c = lane; c < W; c += 32) {
            const float fa = __fsub_rn((float)c, b.Au);
            const float d = __fadd_rn(__fmul_rn(fa, b.cdu), db);
            const float s = __fadd_rn(__fmul_rn(fa, b.csu), sb);
            if (s >= 0.f && s <= 1.f && d >= -half_width && d <= half_width) {
                const double x = (double)as_f32(__ldg(row + c));
                m0 += x;
                m1 += x * (double)d;
            }
        }
    }
    if (p >= 0) {
        m0 = warp_sum(m0);
        m1 = warp_sum(m1);
        if (lane == 0) {
            atomicAdd(moments + 2 * p, m0);
            atomicAdd(moments + 2 * p + 1, m1);
        }
    }
}

// ------------------------------------------------------------------ azimuthal phase

template <class T>
__global__ void k_theta_mean(const T *__restrict__ x, int n_h, int n_t, int n_r, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (ih, ir)
    if (i >= (int64_t)n_h * n_r) return;
    const int ih = (int)(i / n_r), ir = (int)(i - (int64_t)ih * n_r);
    const T *base = x + (int64_t)ih * n_t * n_r + ir;
    double s = 0.0;
    for (int it = 0; it < n_t; ++it) s += (double)as_f32(base[(int64_t)it * n_r]);
    const float m = (float)(s / n_t);
    float *ob = out + (int64_t)ih * n_t * n_r + ir;
    for (int it = 0; it < n_t; ++it) ob[(int64_t)it * n_r] = m;
}

// First-harmonic fits of c = m1 / m0 (0 where m0 = 0) of the scan and of the template,
// both minus the azimuthal mean's: out = phi, amplitude (scan), phi, amplitude (template).
__global__ void __launch_bounds__(32)
k_phase(const double *__restrict__ m_scan, const double *__restrict__ m_tmpl,
        const double *__restrict__ m_mean, const double *__restrict__ angles, int n, double *out)
{
    auto cen = [](const double *m, int i) { return m[2 * i] != 0.0 ? m[2 * i + 1] / m[2 * i] : 0.0; };
    double acc[12];
    for (int q = 0; q < 12; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) {
        const double c = cos(angles[i]), s = sin(angles[i]);
        const double y0 = cen(m_scan, i) - cen(m_mean, i), y1 = cen(m_tmpl, i) - cen(m_mean, i);
        acc[0] += 1.0; acc[1] += c; acc[2] += s; acc[3] += c * c; acc[4] += c * s; acc[5] += s * s;
        acc[6] += y0; acc[7] += c * y0; acc[8] += s * y0;
        acc[9] += y1; acc[10] += c * y1; acc[11] += s * y1;
    }
    for (int q = 0; q < 12; ++q) acc[q] = warp_sum(acc[q]);
    if (threadIdx.x != 0) return;
    for (int f = 0; f < 2; ++f) {
        double cf[3] = {nan(""), nan(""), nan("")};
        solve3(acc, acc + 6 + 3 * f, cf);
        out[2 * f] = atan2(cf[2], cf[1]);
        out[2 * f + 1] = hypot(cf[1], cf[2]);
    }
}

// ------------------------------------------------------------------ host helpers

// Device time of the pose kernels (cyl_pose_set_timing): events around each timed launch
// on its stream, read after the call's own synchronisation.
struct PoseTiming {
    std::mutex mu;
    bool on = false;
    double ms[2] = {0, 0};      // 0: corner pass, 1: Levenberg-Marquardt pass
    int64_t n[2] = {0, 0};
} g_timing;

struct KernelTimer {
    int kind;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KernelTimer(int k, cudaStream_t s) : kind(k), st(s)
    {
        bool on;
        {
            std::lock_guard<std::mutex> l(g_timing.mu);
            on = g_timing.on;
        }
        if (on && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
            cudaEventRecord(e0, st);
    }
    void stop()
    {
        if (e1) cudaEventRecord(e1, st);
    }
    // after the stream has been synchronised
    void collect()
    {
        float ms = 0.f;
        if (e1 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            std::lock_guard<std::mutex> l(g_timing.mu);
            g_timing.ms[kind] += ms;
            g_timing.n[kind] += 1;
        }
    }
    ~KernelTimer()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

struct DevBlob {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBlob()
    {
        if (p) cudaFreeAsync(p, st);
    }
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Device scratch and pinned staging of the synchronous pose calls, one set per host
// thread, grown on demand (freed at thread exit).
struct PoseScratch {
    int dev = -1;
    void *d = nullptr, *h = nullptr;
    size_t dcap = 0, hcap = 0;
    int reserve(int device, size_t dbytes, size_t hbytes)
    {
        if (device != dev) release();
        dev = device;
        if (dcap < dbytes) {
            if (d) cudaFree(d);
            d = nullptr;
            dcap = 0;
            if (cudaMalloc(&d, dbytes) != cudaSuccess) {
                cudaGetLastError();
                return set_error(CYL_ENOMEM, "pose scratch");
            }
            dcap = dbytes;
        }
        if (hcap < hbytes) {
            if (h) cudaFreeHost(h);
            h = nullptr;
            hcap = 0;
            if (cudaMallocHost(&h, hbytes) != cudaSuccess) {
                cudaGetLastError();
                return set_error(CYL_ENOMEM, "pose staging");
            }
            hcap = hbytes;
        }
        return CYL_OK;
    }
    void release()
    {
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        d = h = nullptr;
        dcap = hcap = 0;
    }
    ~PoseScratch() { release(); }
};
thread_local PoseScratch t_scratch;

int persistent_warps()
{
    static int warps = 0;
    if (!warps) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_corners<float>, kCornerThreads, 0);
        warps = std::max(1, sms) * std::max(1, per_sm) * (kCornerThreads / 32);
    }
    return warps;
}

float float_at_or_below(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

void window_of(const cyl_geom &g, const cyl_pose_params &p, int w[4])
{
    if (!p.roi[0] && !p.roi[1] && !p.roi[2] && !p.roi[3]) {
        w[0] = 0; w[1] = g.det_w; w[2] = 0; w[3] = g.det_h;
    } else {
        for (int k = 0; k < 4; ++k) w[k] = p.roi[k];
    }
}

int check_params(const cyl_geom &g, const cyl_pose_params *p)
{
    if (!p) return set_error(CYL_EINVAL, "params is null");
    if (!std::isfinite(p->threshold)) return set_error(CYL_EINVAL, "threshold must be finite");
    if (p->dilate_px < 0 || p->dilate_px > 65535) return set_error(CYL_EINVAL, "dilate_px must be in 0 .. 65535");
    if (!std::isfinite(p->gamma)) return set_error(CYL_EINVAL, "gamma must be finite");
    int w[4];
    window_of(g, *p, w);
    if (w[0] < 0 || w[0] >= w[1] || w[1] > g.det_w || w[2] < 0 || w[2] >= w[3] || w[3] > g.det_h)
        return set_error(CYL_EINVAL, "window must satisfy 0 <= u0 < u1 <= W and 0 <= v0 < v1 <= H");
    return CYL_OK;
}

int check_geom(const cyl_geom *g)
{
    int rc = validate_geom(g);
    if (rc) return rc;
    if (g->det_w > CYL_MAX_DET_SIDE || g->det_h > CYL_MAX_DET_SIDE)
        return set_error(CYL_EINVAL, "det_w and det_h must be <= CYL_MAX_DET_SIDE");
    return CYL_OK;
}

bool valid_dt(int t) { return t == CYL_F32 || t == CYL_F16 || t == CYL_BF16; }

void stage_view_table(const cyl_geom &g, std::vector<ViewLM> &out)
{
    std::vector<ProjGeom> geo;
    const cyl_pose id{0, 0, 0, 0, 0, 0};
    build_views(g, id, geo);
    for (const ProjGeom &v : geo) {
        ViewLM w{};
        for (int k = 0; k < 3; ++k) {
            w.S[k] = v.S[k];
            w.D0[k] = v.D0[k];
            w.du[k] = v.du[k];
            w.dv[k] = v.dv[k];
        }
        double t[3], SD[3] = {v.S[0] - v.D0[0], v.S[1] - v.D0[1], v.S[2] - v.D0[2]};
        cross3(w.du, w.dv, w.n);
        cross3(w.dv, w.n, t);
        const double q1 = dot3(w.du, t);
        for (int k = 0; k < 3; ++k) w.e1[k] = t[k] / q1;
        cross3(w.n, w.du, t);
        const double q2 = dot3(w.dv, t);
        for (int k = 0; k < 3; ++k) w.e2[k] = t[k] / q2;
        w.a0 = dot3(w.e1, SD);
        w.b0 = dot3(w.e2, SD);
        w.c0 = -dot3(w.n, SD);
        w.su = std::sqrt(dot3(w.du, w.du));
        w.sv = std::sqrt(dot3(w.dv, w.dv));
        out.push_back(w);
    }
}

// Pixel coordinates of the stage point X in view w.
void project_host(const ViewLM &w, const double X[3], double &a, double &b)
{
    const double Y[3] = {X[0] - w.S[0], X[1] - w.S[1], X[2] - w.S[2]};
    const double t = w.c0 / dot3(w.n, Y);
    a = w.a0 + t * dot3(w.e1, Y);
    b = w.b0 + t * dot3(w.e2, Y);
}

void band_table(const cyl_geom &g, const cyl_pose &pose, const cyl_band &band, std::vector<BandView> &out)
{
    std::vector<ViewLM> views;
    stage_view_table(g, views);
    double R[3][3];
    alignment_matrix(pose, R);   // X' = R (X - T), so X = R^T X' + T
    double A3[3], B3[3];
    for (int k = 0; k < 3; ++k) {
        A3[k] = R[2][k] * band.h_lo_mm + (k == 0 ? pose.tx : k == 1 ? pose.ty : pose.tz);
        B3[k] = R[2][k] * band.h_hi_mm + (k == 0 ? pose.tx : k == 1 ? pose.ty : pose.tz);
    }
    for (const ViewLM &w : views) {
        double Aa, Ab, Ba, Bb;
        project_host(w, A3, Aa, Ab);
        project_host(w, B3, Ba, Bb);
        const double Lu = (Ba - Aa) * w.su, Lv = (Bb - Ab) * w.sv;
        const double L2 = Lu * Lu + Lv * Lv, L = std::sqrt(L2);
        BandView b;
        b.Au = (float)Aa;
        b.Av = (float)Ab;
        b.cdu = (float)(w.su * Lv / L);
        b.cdv = (float)(-w.sv * Lu / L);
        b.csu = (float)(w.su * Lu / L2);
        b.csv = (float)(w.sv * Lv / L2);
        out.push_back(b);
    }
}

template <class T>
cudaError_t launch_band_t(const void *sino, int n_proj, int W, int H, const BandView *bv, float hw,
                          double *moments, cudaStream_t st)
{
    const int64_t rows = (int64_t)n_proj * H;
    const int64_t per = std::max<int64_t>(1, (rows + persistent_warps() - 1) / persistent_warps());
    const int64_t warps = (rows + per - 1) / per;
    const int blocks = (int)((warps * 32 + kCornerThreads - 1) / kCornerThreads);
    k_band<T><<<blocks, kCornerThreads, 0, st>>>(static_cast<const T *>(sino), n_proj, W, H, bv, hw, per,
                                                 moments);
    return cudaGetLastError();
}

cudaError_t launch_band(const void *sino, cyl_dtype t, int n_proj, int W, int H, const BandView *bv,
                        float hw, double *moments, cudaStream_t st)
{
    switch (t) {
    case CYL_F16: return launch_band_t<__half>(sino, n_proj, W, H, bv, hw, moments, st);
    case CYL_BF16: return launch_band_t<__nv_bfloat16>(sino, n_proj, W, H, bv, hw, moments, st);
    default: return launch_band_t<float>(sino, n_proj, W, H, bv, hw, moments, st);
    }
}

cudaError_t launch_corners(const CornerScan *d_scans, int n_scans, int64_t rows, cyl_dtype t,
                           unsigned long long *keys, unsigned long long *counts, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    const int64_t per = std::max<int64_t>(1, (rows + persistent_warps() - 1) / persistent_warps());
    const int64_t warps = (rows + per - 1) / per;
    const int blocks = (int)((warps * 32 + kCornerThreads - 1) / kCornerThreads);
    switch (t) {
    case CYL_F16:
        k_corners<__half><<<blocks, kCornerThreads, 0, st>>>(d_scans, n_scans, rows, per, keys, counts);
        break;
    case CYL_BF16:
        k_corners<__nv_bfloat16><<<blocks, kCornerThreads, 0, st>>>(d_scans, n_scans, rows, per, keys, counts);
        break;
    default:
        k_corners<float><<<blocks, kCornerThreads, 0, st>>>(d_scans, n_scans, rows, per, keys, counts);
    }
    return cudaGetLastError();
}

CornerScan corner_scan(const cyl_geom &g, const void *sino, cyl_dtype t, const cyl_pose_params &p,
                       int64_t row0, int64_t view0)
{
    CornerScan cs{};
    int w[4];
    window_of(g, p, w);
    cs.sino = sino;
    cs.row0 = row0;
    cs.view0 = view0;
    cs.n_proj = g.n_proj;
    cs.W = g.det_w;
    cs.H = g.det_h;
    cs.u0 = w[0];
    cs.u1 = w[1];
    cs.v0 = w[2];
    cs.v1 = w[3];
    cs.k = p.dilate_px;
    cs.vec = ((uintptr_t)sino % 16 == 0) && ((size_t)g.det_w * dtype_size(t)) % 16 == 0;
    cs.thr = float_at_or_below(p.threshold);
    return cs;
}

#define PO_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);     \
    } while (0)

// Pose estimate of n scans (the body of cyl_estimate_pose[_batch]).
int estimate_poses(int n, const cyl_geom *geoms, const void *const *sinos, cyl_dtype t,
                   const cyl_pose_params *prms, cyl_pose *poses, cyl_pose_info *infos, cudaStream_t st)
{
    std::vector<CornerScan> cscans;
    std::vector<TrackScan> tscans;
    std::vector<ViewLM> views;
    int64_t rows = 0, nviews = 0;
    for (int i = 0; i < n; ++i) {
        cscans.push_back(corner_scan(geoms[i], sinos[i], t, prms[i], rows, nviews));
        TrackScan ts{nviews, geoms[i].n_proj, geoms[i].det_h, prms[i].max_iter > 0 ? prms[i].max_iter : 100,
                     prms[i].gamma};
        tscans.push_back(ts);
        stage_view_table(geoms[i], views);
        rows += (int64_t)geoms[i].n_proj * (cscans.back().v1 - cscans.back().v0);
        nviews += geoms[i].n_proj;
    }
    const size_t o_keys = 0, o_cnt = align_up(o_keys + 32 * nviews), o_cs = align_up(o_cnt + 8 * nviews);
    const size_t o_ts = align_up(o_cs + sizeof(CornerScan) * n), o_vw = align_up(o_ts + sizeof(TrackScan) * n);
    const size_t o_out = align_up(o_vw + sizeof(ViewLM) * nviews);
    const size_t total = align_up(o_out + sizeof(double) * kOutPose * n);
    // this thread's cached scratch: the call ends synchronised, so the next call may reuse it
    int dev = 0;
    PO_CUDA(cudaGetDevice(&dev));
    int rc = t_scratch.reserve(dev, total, total - o_cs);
    if (rc) return rc;
    char *host = static_cast<char *>(t_scratch.h);   // pinned: tables in, results out
    memcpy(host, cscans.data(), sizeof(CornerScan) * n);
    memcpy(host + (o_ts - o_cs), tscans.data(), sizeof(TrackScan) * n);
    memcpy(host + (o_vw - o_cs), views.data(), sizeof(ViewLM) * nviews);
    char *b = static_cast<char *>(t_scratch.d);
    auto *keys = reinterpret_cast<unsigned long long *>(b + o_keys);
    auto *cnts = reinterpret_cast<unsigned long long *>(b + o_cnt);
    PO_CUDA(cudaMemsetAsync(b, 0, o_cs, st));
    PO_CUDA(cudaMemcpyAsync(b + o_cs, host, o_out - o_cs, cudaMemcpyHostToDevice, st));
    KernelTimer tc(0, st);
    PO_CUDA(launch_corners(reinterpret_cast<const CornerScan *>(b + o_cs), n, rows, t, keys, cnts, st));
    tc.stop();
    KernelTimer tt(1, st);
    k_track_pose<<<n, 64, 0, st>>>(reinterpret_cast<const TrackScan *>(b + o_ts),
                                   reinterpret_cast<const ViewLM *>(b + o_vw), keys,
                                   reinterpret_cast<double *>(b + o_out));
    PO_CUDA(cudaGetLastError());
    tt.stop();
    const double *out = reinterpret_cast<const double *>(host + (o_out - o_cs));   // after the tables
    PO_CUDA(cudaMemcpyAsync(host + (o_out - o_cs), b + o_out, sizeof(double) * kOutPose * n, cudaMemcpyDeviceToHost,
                            st));
    PO_CUDA(cudaStreamSynchronize(st));
    tc.collect();
    tt.collect();
    for (int i = 0; i < n; ++i) {
        const double *o = out + (size_t)kOutPose * i;
        if (poses) poses[i] = cyl_pose{o[12], o[13], o[14], o[15], o[16], o[17]};
        if (infos) {
            cyl_pose_info &f = infos[i];
            for (int k = 0; k < 3; ++k) {
                f.top_mm[k] = o[k];
                f.bottom_mm[k] = o[3 + k];
            }
            f.rms_mm[0] = o[6];
            f.rms_mm[1] = o[7];
            f.iters[0] = (int32_t)o[8];
            f.iters[1] = (int32_t)o[9];
            f.n_views = (int32_t)o[10];
            f.status = (int32_t)o[11];
        }
    }
    return CYL_OK;
}

}  // namespace
}  // namespace cylct

using namespace cylct;

extern "C" int cyl_axis_corners(const cyl_geom *geom, const void *sino, cyl_dtype sino_dtype,
                                const cyl_pose_params *params, int32_t *corners_out, int64_t *counts_out,
                                void *stream)
{
    int rc = check_geom(geom);
    if (rc) return rc;
    if ((rc = check_params(*geom, params))) return rc;
    if (!valid_dt(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!sino || !corners_out) return set_error(CYL_EINVAL, "null array");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = geom->n_proj;
    CornerScan cs = corner_scan(*geom, sino, sino_dtype, *params, 0, 0);
    const int64_t rows = (int64_t)n * (cs.v1 - cs.v0);
    const size_t o_cnt = align_up(32 * (size_t)n), o_cs = align_up(o_cnt + 8 * (size_t)n);
    DevBlob blob;
    blob.st = st;
    PO_CUDA(cudaMallocAsync(&blob.p, o_cs + sizeof(CornerScan), st));
    char *b = static_cast<char *>(blob.p);
    auto *keys = reinterpret_cast<unsigned long long *>(b);
    auto *cnts = counts_out ? reinterpret_cast<unsigned long long *>(counts_out)
                            : reinterpret_cast<unsigned long long *>(b + o_cnt);
    PO_CUDA(cudaMemsetAsync(b, 0, o_cs, st));
    if (counts_out) PO_CUDA(cudaMemsetAsync(counts_out, 0, sizeof(int64_t) * n, st));
    PO_CUDA(cudaMemcpyAsync(b + o_cs, &cs, sizeof cs, cudaMemcpyHostToDevice, st));
    PO_CUDA(launch_corners(reinterpret_cast<const CornerScan *>(b + o_cs), 1, rows, sino_dtype, keys, cnts, st));
    k_decode_corners<<<(4 * n + 255) / 256, 256, 0, st>>>(keys, n, geom->det_h, corners_out);
    PO_CUDA(cudaGetLastError());
    return CYL_OK;
}

extern "C" int cyl_track_point(const cyl_geom *geom, const double *track, int32_t max_iter, double *out,
                               void *stream)
{
    int rc = check_geom(geom);
    if (rc) return rc;
    if (!track || !out) return set_error(CYL_EINVAL, "null array");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<ViewLM> views;
    stage_view_table(*geom, views);
    DevBlob blob;
    blob.st = st;
    PO_CUDA(cudaMallocAsync(&blob.p, sizeof(ViewLM) * views.size(), st));
    PO_CUDA(cudaMemcpyAsync(blob.p, views.data(), sizeof(ViewLM) * views.size(), cudaMemcpyHostToDevice, st));
    k_track_one<<<1, 32, 0, st>>>(static_cast<const ViewLM *>(blob.p), geom->n_proj, track,
                                  max_iter > 0 ? max_iter : 100, out);
    PO_CUDA(cudaGetLastError());
    return CYL_OK;
}

extern "C" int cyl_estimate_pose(const cyl_geom *geom, const void *sino, cyl_dtype sino_dtype,
                                 const cyl_pose_params *params, cyl_pose *pose_out, cyl_pose_info *info_out,
                                 void *stream)
{
    int rc = check_geom(geom);
    if (rc) return rc;
    if ((rc = check_params(*geom, params))) return rc;
    if (!valid_dt(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!sino || !pose_out) return set_error(CYL_EINVAL, "null sino or pose_out");
    const void *s[1] = {sino};
    return estimate_poses(1, geom, s, sino_dtype, params, pose_out, info_out, (cudaStream_t)stream);
}

extern "C" int cyl_estimate_pose_batch(int32_t n, const cyl_geom *geoms, const void *const *sinos,
                                       cyl_dtype sino_dtype, const cyl_pose_params *params,
                                       cyl_pose *poses_out, cyl_pose_info *infos_out, void *stream)
{
    if (n < 0 || n > CYL_MAX_BATCH) return set_error(CYL_EINVAL, "n must be in 0 .. CYL_MAX_BATCH");
    if (n == 0) return CYL_OK;
    if (!geoms || !sinos || !params || !poses_out) return set_error(CYL_EINVAL, "null array");
    if (!valid_dt(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    for (int i = 0; i < n; ++i) {
        int rc = check_geom(&geoms[i]);
        if (rc) return rc;
        if ((rc = check_params(geoms[i], &params[i]))) return rc;
        if (!sinos[i]) return set_error(CYL_EINVAL, "null sinogram");
    }
    return estimate_poses(n, geoms, sinos, sino_dtype, params, poses_out, infos_out, (cudaStream_t)stream);
}

extern "C" int cyl_band_moments(const cyl_geom *geom, const cyl_pose *pose, const void *sino,
                                cyl_dtype sino_dtype, const cyl_band *band, double *moments_out, void *stream)
{
    int rc = validate_geom(geom);
    if (rc) return rc;
    if (!pose || !band) return set_error(CYL_EINVAL, "null pose or band");
    if (!(band->h_lo_mm < band->h_hi_mm) || !std::isfinite(band->h_lo_mm) || !std::isfinite(band->h_hi_mm) ||
        !(band->half_width_mm > 0.0) || !std::isfinite(band->half_width_mm))
        return set_error(CYL_EINVAL, "band needs finite h_lo < h_hi and half_width > 0");
    if (!valid_dt(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!sino || !moments_out) return set_error(CYL_EINVAL, "null array");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BandView> bv;
    band_table(*geom, *pose, *band, bv);
    DevBlob blob;
    blob.st = st;
    PO_CUDA(cudaMallocAsync(&blob.p, sizeof(BandView) * bv.size(), st));
    PO_CUDA(cudaMemcpyAsync(blob.p, bv.data(), sizeof(BandView) * bv.size(), cudaMemcpyHostToDevice, st));
    PO_CUDA(cudaMemsetAsync(moments_out, 0, sizeof(double) * 2 * geom->n_proj, st));
    PO_CUDA(launch_band(sino, sino_dtype, geom->n_proj, geom->det_w, geom->det_h,
                        static_cast<const BandView *>(blob.p), (float)band->half_width_mm, moments_out, st));
    return CYL_OK;
}

namespace {
double wrap_angle(double x) { return std::atan2(std::sin(x), std::cos(x)); }
double inplane(double psi, double alpha, double beta)
{
    return std::atan2(std::sin(psi - alpha), std::cos(beta) * std::cos(psi - alpha));
}
}  // namespace

extern "C" int cyl_gamma_from_phase(double phi_p, double phi_p_ref, double alpha, double beta,
                                    double gamma_ref, double *gamma_out)
{
    if (!gamma_out) return set_error(CYL_EINVAL, "gamma_out is null");
    if (!std::isfinite(phi_p) || !std::isfinite(phi_p_ref) || !std::isfinite(alpha) || !std::isfinite(beta) ||
        !std::isfinite(gamma_ref))
        return set_error(CYL_EINVAL, "non-finite argument");
    const double phi_g = 0.5 * kPi;
    *gamma_out = wrap_angle(gamma_ref + inplane(phi_g - phi_p, alpha, beta) - inplane(phi_g - phi_p_ref, alpha, beta));
    return CYL_OK;
}

extern "C" int cyl_estimate_gamma(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, const void *tmpl,
                                  cyl_dtype tmpl_dtype, const cyl_band *band, int32_t passes, double *gamma_out,
                                  double *diag_out, void *stream)
{
    if (!plan || !band || !gamma_out) return set_error(CYL_EINVAL, "null plan, band or gamma_out");
    if (plan->geom.frames_mm) return set_error(CYL_EINVAL, "the phase needs a circular geometry");
    if (!valid_dt(sino_dtype) || !valid_dt(tmpl_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!sino || !tmpl) return set_error(CYL_EINVAL, "null array");
    if (passes < 1 || passes > 16) return set_error(CYL_EINVAL, "passes must be in 1 .. 16");
    if (!(band->h_lo_mm < band->h_hi_mm) || !std::isfinite(band->h_lo_mm) || !std::isfinite(band->h_hi_mm) ||
        !(band->half_width_mm > 0.0) || !std::isfinite(band->half_width_mm))
        return set_error(CYL_EINVAL, "band needs finite h_lo < h_hi and half_width > 0");
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != plan->device) cudaSetDevice(plan->device);
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{dev_prev};
    std::lock_guard<std::mutex> lock(plan->mu);
    const int n = plan->geom.n_proj;
    const size_t nq = (size_t)n * plan->n_pix;
    std::vector<BandView> bv;   // the band follows the axis, which a spin leaves in place
    band_table(plan->geom, plan->pose, *band, bv);
    const size_t o_mean = 0, o_q = align_up(sizeof(float) * plan->n_vox);
    const size_t o_m = align_up(o_q + sizeof(float) * 2 * nq), o_ang = align_up(o_m + sizeof(double) * 6 * n);
    const size_t o_bv = align_up(o_ang + sizeof(double) * n), o_out = align_up(o_bv + sizeof(BandView) * n);
    const size_t total = align_up(o_out + 4 * sizeof(double));
    int rc = plan->ensure(&plan->d_gamma, plan->gamma_cap, total);
    if (rc) return rc;
    char *b = static_cast<char *>(plan->d_gamma);
    float *mean = reinterpret_cast<float *>(b + o_mean);
    float *q_tmpl = reinterpret_cast<float *>(b + o_q), *q_mean = q_tmpl + nq;
    double *m = reinterpret_cast<double *>(b + o_m);
    const BandView *d_bv = reinterpret_cast<const BandView *>(b + o_bv);
    cudaStream_t user = (cudaStream_t)stream, ws = plan->ws;
    PO_CUDA(cudaEventRecord(plan->ev_in, user));
    PO_CUDA(cudaStreamWaitEvent(ws, plan->ev_in, 0));
    PO_CUDA(cudaMemcpyAsync(b + o_ang, plan->angles.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ws));
    PO_CUDA(cudaMemcpyAsync(b + o_bv, bv.data(), sizeof(BandView) * n, cudaMemcpyHostToDevice, ws));
    PO_CUDA(cudaMemsetAsync(m, 0, sizeof(double) * 6 * n, ws));
    const GridDev &g = plan->g;
    const int64_t hr = (int64_t)g.n_h * g.n_r;
    const int tb = 256, nb = (int)((hr + tb - 1) / tb);
    switch (tmpl_dtype) {
    case CYL_F16: k_theta_mean<<<nb, tb, 0, ws>>>(static_cast<const __half *>(tmpl), g.n_h, g.n_t, g.n_r, mean); break;
    case CYL_BF16:
        k_theta_mean<<<nb, tb, 0, ws>>>(static_cast<const __nv_bfloat16 *>(tmpl), g.n_h, g.n_t, g.n_r, mean);
        break;
    default: k_theta_mean<<<nb, tb, 0, ws>>>(static_cast<const float *>(tmpl), g.n_h, g.n_t, g.n_r, mean);
    }
    PO_CUDA(cudaGetLastError());
    const float hw = (float)band->half_width_mm;
    // spin-independent: the scan's moments and the azimuthal mean's projection
    PO_CUDA(cudaMemsetAsync(q_mean, 0, sizeof(float) * nq, ws));   // rays that miss the grid stay 0
    PO_CUDA(launch_fp_rays(plan->scan_dev(), plan->p_fp, 0, n, mean, CYL_F32, q_mean, nullptr, 0, ws,
                           plan->ray_list()));
    PO_CUDA(launch_band(sino, sino_dtype, n, g.det_w, g.det_h, d_bv, hw, m, ws));
    PO_CUDA(launch_band(q_mean, CYL_F32, n, g.det_w, g.det_h, d_bv, hw, m + 4 * n, ws));
    double out[4] = {0, 0, 0, 0}, gamma = plan->pose.gamma;
    for (int pass = 0; pass < passes; ++pass) {
        if (pass > 0) {   // the template's spin moves to the current estimate
            cyl_pose ps = plan->pose;
            ps.gamma = gamma;
            if ((rc = plan->upload_pose(ps, ws))) return rc;
        }
        PO_CUDA(cudaMemsetAsync(q_tmpl, 0, sizeof(float) * nq, ws));
        PO_CUDA(cudaMemsetAsync(m + 2 * n, 0, sizeof(double) * 2 * n, ws));
        PO_CUDA(launch_fp_rays(plan->scan_dev(), plan->p_fp, 0, n, tmpl, tmpl_dtype, q_tmpl, nullptr, 0, ws,
                               plan->ray_list()));
        PO_CUDA(launch_band(q_tmpl, CYL_F32, n, g.det_w, g.det_h, d_bv, hw, m + 2 * n, ws));
        k_phase<<<1, 32, 0, ws>>>(m, m + 2 * n, m + 4 * n, reinterpret_cast<const double *>(b + o_ang), n,
                                  reinterpret_cast<double *>(b + o_out));
        PO_CUDA(cudaGetLastError());
        PO_CUDA(cudaMemcpyAsync(out, b + o_out, sizeof out, cudaMemcpyDeviceToHost, ws));
        PO_CUDA(cudaStreamSynchronize(ws));
        double next;
        if ((rc = cyl_gamma_from_phase(out[0], out[2], plan->pose.alpha, plan->pose.beta, plan->pose.gamma, &next)))
            return rc;
        gamma = next;
    }
    if (passes > 1 || gamma != plan->pose.gamma) {   // leave the plan posed with the estimate
        cyl_pose ps = plan->pose;
        ps.gamma = gamma;
        if ((rc = plan->upload_pose(ps, ws))) return rc;
    }
    PO_CUDA(cudaEventRecord(plan->ev_out, ws));
    PO_CUDA(cudaStreamWaitEvent(user, plan->ev_out, 0));
    if (diag_out) memcpy(diag_out, out, sizeof out);
    *gamma_out = gamma;
    return CYL_OK;
}

extern "C" int cyl_pose_set_timing(int enable)
{
    std::lock_guard<std::mutex> l(g_timing.mu);
    g_timing.on = enable != 0;
    for (int k = 0; k < 2; ++k) {
        g_timing.ms[k] = 0.0;
        g_timing.n[k] = 0;
    }
    return CYL_OK;
}

extern "C" int cyl_pose_kernel_time(int kind, double *ms_total, int64_t *launches)
{
    if (kind < 0 || kind > 1) return set_error(CYL_EINVAL, "kind must be 0 or 1");
    std::lock_guard<std::mutex> l(g_timing.mu);
    if (ms_total) *ms_total = g_timing.ms[kind];
    if (launches) *launches = g_timing.n[kind];
    return CYL_OK;
}
