// Exact ray traversal of the cylindrical grid (device code).
//
// t_jl of Sec. 2.2 (Eq. 5) is the length of ray j inside voxel l.  A voxel of the grid of
// Eq. 2 is bounded by two radial shells, two azimuthal wedge half-planes and two axial
// slab planes, so a ray's row of the system matrix is the list of pieces between
// consecutive crossings of those three families.  Each ray walks them incrementally: it
// keeps the next crossing of each family and always advances the nearest one, so the
// voxel index changes by one step of one family at a time.
//
// Parametrisation.  u is the distance (mm) along the ray from its closest approach P* to
// the z' axis.  With a = e_x^2 + e_y^2 and d the axis distance,
//     r(u)^2 = a u^2 + d^2,   so shell k is crossed at u = -+sqrt((r_k^2 - d^2) / a);
//     theta(u) is monotone (sense = sign of (P* x e)_z); wedge boundary k is crossed at
//     u = -(n_k . P*) / (n_k . e), n_k = (-sin theta_k, cos theta_k), and only on the
//     theta_k half-plane, i.e. when sense * (n_k . e) > 0;
//     h(u) = z* + u e_z, slab plane k is crossed at u = (h_k - z*) / e_z.
// Measuring u from P* keeps positions small (|u| <~ R), so the walk runs in FP32.  The
// ray set-up (clip to the grid cylinder, P*, axis distance, row sum, and the one shell
// crossing that can be near-tangent: the innermost boundary the ray reaches) runs once
// per ray in FP64 and is stored as a 48-byte record.
//
// Tiles.  The volume is cut into tiles of TT wedges x TH slabs x all shells; a tile is a
// sector prism (angle <= pi/2, or the full circle when one tile spans all wedges).  A
// ray's part inside a tile is its clipped interval intersected with the tile's slab
// range and wedge range; the walk inside a tile stops at the tile's own boundaries.
// The boundary positions use the same expressions as the crossings, so the pieces a ray
// leaves in the tiles it crosses are the pieces of its whole row.
//
// Robustness: every crossing is clamped to be >= the current position and every index
// change is a single step, so rounding near a boundary only creates a zero-length piece.
// Indices never leave the tile (its exits are the clip, not crossings), and a walk stops
// after max_steps pieces.
//
// Work distribution (tile_walk_all): a warp tests 32 candidate pixels of a tile at once,
// and moves the rays that cross the tile into its idle lanes with shuffles; all lanes
// then step their rays in lock-step, and the warp refills when half of its lanes are
// idle.  Candidates that miss the tile therefore never hold a lane while others walk.
#pragma once

#include "cylct_internal.h"

namespace cylct {

constexpr float kInf = 3.0e38f;
constexpr float kTwoPiF = 6.283185307179586f;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kRefillBelow = 16;   // refill a warp once this many lanes or fewer walk
constexpr int kStepsPerCheck = 2;  // steps between two refill checks

// FP32 ray record, computed once per plan and pose in FP64 (k_rays).
//   a = (P*x, P*y, P*z, utan)   utan: |u| of shell boundary kstar
//   b = (e_x, e_y, e_z, d^2)
//   c = (u_in, u_out, L, kstar) L: chord in the grid cylinder (row sum of Eq. 6);
//                               u_in > u_out marks a ray that misses the grid;
//                               kstar = -1 marks a ray parallel to the axis.
struct RayRec {
    float4 a, b, c;
};

__device__ __forceinline__ float fsqrt_fast(float x)
{
    return x > 0.f ? x * rsqrtf(x) : 0.f;
}

// FP64 set-up of ray (p, iu, iv) into a record.
__device__ __forceinline__ RayRec setup_ray(const GridDev &g, const ProjGeom &pg, int iu, int iv)
{
    RayRec rr;
    rr.a = make_float4(0.f, 0.f, 0.f, 0.f);
    rr.b = make_float4(0.f, 0.f, 0.f, 0.f);
    rr.c = make_float4(1.f, 0.f, 0.f, __int_as_float(0));   // miss
    double Sx = pg.S[0], Sy = pg.S[1], Sz = pg.S[2];
    double dx = pg.D0[0] + iu * pg.du[0] + iv * pg.dv[0] - Sx;
    double dy = pg.D0[1] + iu * pg.du[1] + iv * pg.dv[1] - Sy;
    double dz = pg.D0[2] + iu * pg.du[2] + iv * pg.dv[2] - Sz;
    double len = sqrt(dx * dx + dy * dy + dz * dz);
    double inv_len = 1.0 / len;
    double ex = dx * inv_len, ey = dy * inv_len, ez = dz * inv_len;
    double a = ex * ex + ey * ey;
    double R = g.radius, half = 0.5 * g.height;
    double s_lo, s_hi, sstar, d2, inv_a = 0.0;
    bool radial = a > 1e-18;
    if (radial) {
        inv_a = 1.0 / a;
        double m = Sx * ey - Sy * ex;            // (S x e)_z, so a d^2 = m^2
        d2 = m * m * inv_a;
        if (d2 >= R * R) return rr;
        sstar = -(Sx * ex + Sy * ey) * inv_a;
        double hR = sqrt((R * R - d2) * inv_a);
        s_lo = fmax(sstar - hR, 0.0);
        s_hi = fmin(sstar + hR, len);
    } else {                                      // parallel to the axis
        d2 = Sx * Sx + Sy * Sy;
        if (d2 > R * R) return rr;
        sstar = 0.0;
        s_lo = 0.0;
        s_hi = len;
    }
    if (ez != 0.0) {
        double iz = 1.0 / ez;
        double s1 = (-half - Sz) * iz, s2 = (half - Sz) * iz;
        s_lo = fmax(s_lo, fmin(s1, s2));
        s_hi = fmin(s_hi, fmax(s1, s2));
    } else if (Sz < -half || Sz > half) {
        return rr;
    }
    if (!(s_hi > s_lo)) return rr;
    int ks = 0;
    float utan = 0.f;
    if (radial) {
        ks = (int)floor(sqrt(d2) / g.dr_d) + 1;
        if (ks < g.n_r) {
            double rk = ks * g.dr_d;
            utan = (float)sqrt(fmax(rk * rk - d2, 0.0) * inv_a);
        }
    } else {
        ks = -1;
    }
    rr.a = make_float4((float)(Sx + sstar * ex), (float)(Sy + sstar * ey), (float)(Sz + sstar * ez),
                       utan);
    rr.b = make_float4((float)ex, (float)ey, (float)ez, (float)d2);
    rr.c = make_float4((float)(s_lo - sstar), (float)(s_hi - sstar), (float)(s_hi - s_lo),
                       __int_as_float(ks));
    return rr;
}

// Tile of the volume: wedges [t0, t1), slabs [s0, s1), all shells.
struct Tile {
    int t0, t1, s0, s1;
    bool full_circle;       // spans all wedges: wedge index wraps, no wedge clip
};

__device__ __forceinline__ Tile tile_of(const TileDev &td, const GridDev &g, int tile)
{
    Tile t;
    const int tt = tile % td.n_tt, ht = tile / td.n_tt;
    t.t0 = tt * td.tt;
    t.t1 = min(t.t0 + td.tt, g.n_t);
    t.s0 = ht * td.th;
    t.s1 = min(t.s0 + td.th, g.n_h);
    t.full_circle = td.n_tt == 1;
    return t;
}

// Interval [ua, ub] of a ray inside a tile; false if empty.
__device__ __forceinline__ bool clip_tile(const GridDev &g, const float2 *__restrict__ trig,
                                          const RayRec &rr, const Tile &t, float &ua_out,
                                          float &ub_out)
{
    float ua = rr.c.x, ub = rr.c.y;
    if (!(ub > ua)) return false;
    const float px = rr.a.x, py = rr.a.y, pz = rr.a.z;
    const float ex = rr.b.x, ey = rr.b.y, ez = rr.b.z;
    const bool radial = __float_as_int(rr.c.w) >= 0;
    if (ez != 0.f) {
        const float inv_ez = 1.f / ez;
        const float c0 = (g.h0 - pz) * inv_ez, c1 = g.dh * inv_ez;
        const float h_lo = fmaf((float)t.s0, c1, c0), h_hi = fmaf((float)t.s1, c1, c0);
        ua = fmaxf(ua, fminf(h_lo, h_hi));
        ub = fminf(ub, fmaxf(h_lo, h_hi));
    } else {
        const float hz = pz - g.h0;
        if (hz < t.s0 * g.dh || hz > t.s1 * g.dh) return false;
    }
    if (!t.full_circle && radial) {
        // a sector of angle <= pi/2: left of theta_t0 (n_a . P >= 0) and right of
        // theta_t1 (n_b . P <= 0)
        const float2 ca = trig[t.t0], cb = trig[t.t1 == g.n_t ? 0 : t.t1];
        const float nda = ca.x * ey - ca.y * ex, noa = ca.x * py - ca.y * px;
        const float ndb = cb.x * ey - cb.y * ex, nob = cb.x * py - cb.y * px;
        if (nda != 0.f) {
            const float ux = __fdividef(-noa, nda);
            if (nda > 0.f) ua = fmaxf(ua, ux); else ub = fminf(ub, ux);
        } else if (noa < 0.f) {
            return false;
        }
        if (ndb != 0.f) {
            const float ux = __fdividef(-nob, ndb);
            if (ndb < 0.f) ua = fmaxf(ua, ux); else ub = fminf(ub, ux);
        } else if (nob > 0.f) {
            return false;
        }
    } else if (!t.full_circle) {
        // parallel to the axis: one wedge for the whole ray
        float th = atan2f(py, px);
        th = th < 0.f ? th + kTwoPiF : th;
        const int it = min((int)(th * g.inv_dth), g.n_t - 1);
        if (it < t.t0 || it >= t.t1) return false;
    }
    ua_out = ua;
    ub_out = ub;
    return ub > ua;
}

// State of one ray walking through one tile.  Each family keeps the index of the next
// boundary it will cross and the direction it moves in:
//   shells: kr, sdir (-1 while moving inward, +1 outward); the crossing of shell k is at
//           u = sdir * sqrt(A k^2 + B), A = dr^2 / a, B = -d^2 / a (utan for k = kstar);
//   wedges: kt, ccw; crossing at -(n_kt . P*) / (n_kt . e);
//   slabs:  kh, hdir; crossing at c0 + kh c1.
struct Walker {
    float px, py, ex, ey, A, B, utan, c0, c1;
    float u, ub, ur, ut, uh;
    int idx, it, kr, kt, kh, kstar, sdir, hdir, hstride, steps;
    bool ccw;

    __device__ __forceinline__ float shell_u(const GridDev &g) const
    {
        if (kr >= g.n_r) return kInf;
        const float kf = (float)kr;
        const float q = (kr == kstar) ? utan : fsqrt_fast(fmaxf(fmaf(A * kf, kf, B), 0.f));
        return fmaxf(sdir < 0 ? -q : q, u);
    }
    __device__ __forceinline__ float wedge_u(const float2 *__restrict__ trig, const Tile &t) const
    {
        if (kt < 0) return kInf;
        const float2 cs = trig[kt];
        const float nd = cs.x * ey - cs.y * ex;
        if (ccw ? nd <= 0.f : nd >= 0.f) return kInf;
        const float no = cs.x * py - cs.y * px;
        return fmaxf(__fdividef(-no, nd), u);
    }
    __device__ __forceinline__ float slab_u(const Tile &t) const
    {
        return (hdir != 0 && kh > t.s0 && kh < t.s1) ? fmaxf(fmaf((float)kh, c1, c0), u) : kInf;
    }
    // next wedge boundary after entering wedge it (-1: none inside the tile)
    __device__ __forceinline__ int wedge_next(const GridDev &g, const Tile &t, int it_) const
    {
        if (g.n_t == 1) return -1;
        if (ccw) {
            const int k = it_ + 1;
            if (!t.full_circle && k >= t.t1) return -1;
            return k == g.n_t ? 0 : k;
        }
        if (!t.full_circle && it_ <= t.t0) return -1;
        return it_;
    }

    // Start at the tile entry ua of ray rr; the walk ends at ub.
    __device__ __forceinline__ void init(const GridDev &g, const float2 *__restrict__ trig,
                                         const Tile &t, const RayRec &rr, float ua, float ub_)
    {
        px = rr.a.x;
        py = rr.a.y;
        const float pz = rr.a.z;
        ex = rr.b.x;
        ey = rr.b.y;
        const float ez = rr.b.z;
        utan = rr.a.w;
        kstar = __float_as_int(rr.c.w);
        const bool radial = kstar >= 0;
        const float inv_a = radial ? 1.f / fmaf(ex, ex, ey * ey) : 0.f;
        A = g.dr * g.dr * inv_a;
        B = -rr.b.w * inv_a;
        const float inv_ez = ez != 0.f ? 1.f / ez : 0.f;
        c0 = (g.h0 - pz) * inv_ez;
        c1 = g.dh * inv_ez;
        ccw = (px * ey - py * ex) >= 0.f;
        u = ua;
        ub = ub_;
        steps = 0;
        const float x = fmaf(u, ex, px), y = fmaf(u, ey, py), z = fmaf(u, ez, pz);
        const int ir = min((int)(sqrtf(fmaf(x, x, y * y)) * g.inv_dr), g.n_r - 1);
        float th = atan2f(y, x);
        if (t.full_circle) {
            th = th < 0.f ? th + kTwoPiF : th;
            it = min((int)(th * g.inv_dth), g.n_t - 1);
        } else {
            // angle from the tile's first boundary, wrapped to [-pi, pi): a point just
            // below theta = 2 pi belongs to a tile starting at 0 (tiles span <= pi/2)
            float rel = th - (float)t.t0 * g.dth;
            rel = rel < -0.5f * kTwoPiF ? rel + kTwoPiF : (rel >= 0.5f * kTwoPiF ? rel - kTwoPiF : rel);
            it = t.t0 + min(max((int)floorf(rel * g.inv_dth), 0), t.t1 - t.t0 - 1);
        }
        const int ih = min(max((int)floorf((z - g.h0) * g.inv_dh), t.s0), t.s1 - 1);
        const int tw = t.t1 - t.t0;
        hstride = tw * g.n_r;
        idx = ((ih - t.s0) * tw + (it - t.t0)) * g.n_r + ir;
        if (!radial) {
            kr = g.n_r;
            sdir = 1;
            kt = -1;
        } else {
            if (u < 0.f && ir >= kstar) { kr = ir; sdir = -1; }
            else { kr = ir + 1; sdir = 1; }
            kt = wedge_next(g, t, it);
        }
        hdir = ez > 0.f ? 1 : (ez < 0.f ? -1 : 0);
        kh = hdir > 0 ? ih + 1 : ih;
        ur = shell_u(g);
        ut = wedge_u(trig, t);
        uh = slab_u(t);
    }

    // One piece: calls op(idx, length); returns false once the ray has left the tile.
    // Branch-free: the index update and next crossing of all three families are
    // evaluated and the one of the family that moved is kept, so the lanes of a warp
    // never split over which family they advance.
    template <class Op>
    __device__ __forceinline__ bool step(const GridDev &g, const float2 *__restrict__ trig,
                                         const Tile &t, Op &op)
    {
        const float un = fminf(fminf(ur, ut), uh);
        op(idx, fminf(un, ub) - u);
        if (un >= ub || ++steps >= g.max_steps) return false;
        u = un;
        const bool isr = un == ur;
        const bool ist = !isr && un == ut;
        const bool ish = !isr && !ist;
        // shells: inward until kstar, then outward (turnaround re-crosses kstar)
        const int kr2 = sdir > 0 ? kr + 1 : (kr > kstar ? kr - 1 : kr);
        const int sdir2 = (sdir < 0 && kr <= kstar) ? 1 : sdir;
        // wedges: enter wedge it2, next boundary kt2 (-1: none inside the tile)
        int it2 = ccw ? kt : kt - 1;
        it2 = it2 < 0 ? it2 + g.n_t : it2;
        int kc = it2 + 1;
        const bool stop_c = !t.full_circle && kc >= t.t1;
        kc = kc == g.n_t ? 0 : kc;
        const bool stop_w = !t.full_circle && it2 <= t.t0;
        const int kt2 = ccw ? (stop_c ? -1 : kc) : (stop_w ? -1 : it2);
        idx += isr ? sdir : (ist ? (it2 - it) * g.n_r : hdir * hstride);
        kr = isr ? kr2 : kr;
        sdir = isr ? sdir2 : sdir;
        it = ist ? it2 : it;
        kt = ist ? kt2 : kt;
        kh = ish ? kh + hdir : kh;
        const float kf = (float)kr;
        const float qs = (kr == kstar) ? utan : fsqrt_fast(fmaxf(fmaf(A * kf, kf, B), 0.f));
        const float urn = kr >= g.n_r ? kInf : fmaxf(sdir < 0 ? -qs : qs, u);
        const float2 cs = trig[max(kt, 0)];
        const float nd = cs.x * ey - cs.y * ex, no = cs.x * py - cs.y * px;
        const bool okw = kt >= 0 && (ccw ? nd > 0.f : nd < 0.f);
        const float utn = okw ? fmaxf(__fdividef(-no, nd), u) : kInf;
        const float uhn = (hdir != 0 && kh > t.s0 && kh < t.s1) ? fmaxf(fmaf((float)kh, c1, c0), u) : kInf;
        ur = isr ? urn : ur;
        ut = ist ? utn : ut;
        uh = ish ? uhn : uh;
        return true;
    }
};

// Walk every ray of one view whose candidate pixel (inside box bb) crosses tile t.
// ra/rb/rc point at the view's ray records.  K provides:
//   float payload(int64_t j, const RayRec &rr)  per candidate ray j (loads overlap the
//                                               record loads), the ray's start value
//   void piece(int idx, float len, float &acc)  per piece (acc starts at the payload)
//   void end(int64_t j, float acc)              per ray, after its last piece
// s_chunk: a shared int the caller zeroed (chunk counter of this view), s_map: 32 ints
// of shared memory per warp.
template <class K, class W = Walker>
__device__ __forceinline__ void tile_walk_all(const GridDev &g, const float2 *__restrict__ trig,
                                              const Tile &t, const float4 *__restrict__ ra,
                                              const float4 *__restrict__ rb,
                                              const float4 *__restrict__ rc, int4 bb,
                                              K &k, int *s_chunk, int *s_map)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int bw = bb.z - bb.x + 1;
    const int nc = bw * (bb.w - bb.y + 1);
    const int n_chunks = (nc + 31) >> 5;
    int chunk = 0, pos = 32;                // current chunk of 32 candidates, next offset
    bool active = false, more = true;
    W w;
    int64_t j = 0;
    float acc = 0.f;
    auto piece = [&](int idx, float len) { k.piece(idx, len, acc); };
    for (;;) {
        unsigned amask = __ballot_sync(kFull, active);
        // refill: fill every idle lane, testing candidates 32 at a time
        if (__popc(amask) <= kRefillBelow && more) {
            while (amask != kFull && more) {
                if (pos >= 32) {
                    int c0 = 0;
                    if (lane == 0) c0 = atomicAdd(s_chunk, 1);
                    chunk = __shfl_sync(kFull, c0, 0);
                    pos = 0;
                    if (chunk >= n_chunks) {
                        more = false;
                        break;
                    }
                }
                const int c = chunk * 32 + lane;
                bool hit = false;
                RayRec rr;
                float ua = 0.f, ub = 0.f, pay = 0.f;
                int64_t jc = 0;
                if (lane >= pos && c < nc) {
                    jc = (int64_t)(bb.y + c / bw) * g.det_w + (bb.x + c % bw);
                    rr.a = __ldg(ra + jc);
                    rr.b = __ldg(rb + jc);
                    rr.c = __ldg(rc + jc);
                    pay = k.payload(jc, rr);
                    hit = clip_tile(g, trig, rr, t, ua, ub);
                }
                const unsigned hmask = __ballot_sync(kFull, hit);
                const unsigned emask = ~amask;
                const int n_hit = __popc(hmask);
                const int n_take = min(n_hit, __popc(emask));
                if (hit) s_map[__popc(hmask & lt_mask)] = lane;
                __syncwarp();
                const int er = __popc(emask & lt_mask);
                const bool take = !active && er < n_take;
                const int src = take ? s_map[er] : lane;
                pos = n_take < n_hit ? s_map[n_take] : 32;
                __syncwarp();
                RayRec rx;
                rx.a.x = __shfl_sync(kFull, rr.a.x, src);
                rx.a.y = __shfl_sync(kFull, rr.a.y, src);
                rx.a.z = __shfl_sync(kFull, rr.a.z, src);
                rx.a.w = __shfl_sync(kFull, rr.a.w, src);
                rx.b.x = __shfl_sync(kFull, rr.b.x, src);
                rx.b.y = __shfl_sync(kFull, rr.b.y, src);
                rx.b.z = __shfl_sync(kFull, rr.b.z, src);
                rx.b.w = __shfl_sync(kFull, rr.b.w, src);
                rx.c.x = __shfl_sync(kFull, rr.c.x, src);
                rx.c.y = __shfl_sync(kFull, rr.c.y, src);
                rx.c.z = __shfl_sync(kFull, rr.c.z, src);
                rx.c.w = __shfl_sync(kFull, rr.c.w, src);
                const float uax = __shfl_sync(kFull, ua, src);
                const float ubx = __shfl_sync(kFull, ub, src);
                const long long jx = __shfl_sync(kFull, (long long)jc, src);
                const float payx = __shfl_sync(kFull, pay, src);
                if (take) {
                    w.init(g, trig, t, rx, uax, ubx);
                    j = jx;
                    acc = payx;
                    active = true;
                }
                amask = __ballot_sync(kFull, active);
            }
        }
        if (amask == 0) {
            if (!more) break;
            continue;
        }
#pragma unroll
        for (int r = 0; r < kStepsPerCheck; ++r)
            if (active && !w.step(g, trig, t, piece)) {
                k.end(j, acc);
                active = false;
            }
    }
}

}  // namespace cylct
