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
#pragma once

#include "cylct_internal.h"

namespace cylct {

constexpr float kInf = 3.0e38f;
constexpr float kTwoPiF = 6.283185307179586f;

// FP32 ray record, computed once per plan and pose in FP64 (k_rays).
//   a = (P*x, P*y, P*z, utan)   utan: |u| of shell boundary kstar
//   b = (e_x, e_y, e_z, d^2)
//   c = (u_in, u_out, L, kstar) L: chord in the grid cylinder (row sum of Eq. 6);
//                               u_in > u_out marks a ray that misses the grid.
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
        ks = -1;                                  // marks "no shell / wedge crossings"
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

// Walk the pieces of ray rr inside tile t, calling op(local_index, length) for each,
// local_index = ((ih - s0) * (t1 - t0) + (it - t0)) * N_r + ir.  Returns false if the
// ray does not cross the tile.
template <class Op>
__device__ __forceinline__ bool walk_tile(const GridDev &g, const float2 *__restrict__ trig,
                                          const RayRec &rr, const Tile &t, Op &op)
{
    float ua = rr.c.x, ub = rr.c.y;
    if (!(ub > ua)) return false;
    const float px = rr.a.x, py = rr.a.y, pz = rr.a.z;
    const float ex = rr.b.x, ey = rr.b.y, ez = rr.b.z;
    const int kstar = __float_as_int(rr.c.w);
    const bool radial = kstar >= 0;
    const int n_r = g.n_r, n_t = g.n_t;

    // slab range of the tile
    const float inv_ez = ez != 0.f ? 1.f / ez : 0.f;
    const float c0 = (g.h0 - pz) * inv_ez, c1 = g.dh * inv_ez;
    if (ez != 0.f) {
        float h_lo = fmaf((float)t.s0, c1, c0), h_hi = fmaf((float)t.s1, c1, c0);
        ua = fmaxf(ua, fminf(h_lo, h_hi));
        ub = fminf(ub, fmaxf(h_lo, h_hi));
    } else {
        float hz = pz - g.h0;
        if (hz < t.s0 * g.dh || hz > t.s1 * g.dh) return false;
    }
    // wedge range of the tile (a sector of angle <= pi/2: two half-planes)
    const float sense = (px * ey - py * ex) >= 0.f ? 1.f : -1.f;
    const bool ccw = sense > 0.f;
    if (!t.full_circle && radial) {
        float2 ca = trig[t.t0], cb = trig[t.t1 == n_t ? 0 : t.t1];
        // left of theta_t0: n_a . P >= 0
        float nda = ca.x * ey - ca.y * ex, noa = ca.x * py - ca.y * px;
        // right of theta_t1: n_b . P <= 0
        float ndb = cb.x * ey - cb.y * ex, nob = cb.x * py - cb.y * px;
        if (nda != 0.f) {
            float ux = __fdividef(-noa, nda);
            if (nda > 0.f) ua = fmaxf(ua, ux); else ub = fminf(ub, ux);
        } else if (noa < 0.f) {
            return false;
        }
        if (ndb != 0.f) {
            float ux = __fdividef(-nob, ndb);
            if (ndb < 0.f) ua = fmaxf(ua, ux); else ub = fminf(ub, ux);
        } else if (nob > 0.f) {
            return false;
        }
    } else if (!t.full_circle) {
        // parallel to the axis: one wedge for the whole ray
        float th = atan2f(py, px);
        th = th < 0.f ? th + kTwoPiF : th;
        int it = min((int)(th * g.inv_dth), n_t - 1);
        if (it < t.t0 || it >= t.t1) return false;
    }
    if (!(ub > ua)) return false;

    // entry indices
    float u = ua;
    float x = fmaf(u, ex, px), y = fmaf(u, ey, py), z = fmaf(u, ez, pz);
    int ir = min((int)(sqrtf(fmaf(x, x, y * y)) * g.inv_dr), n_r - 1);
    float th = atan2f(y, x);
    int it;
    if (t.full_circle) {
        th = th < 0.f ? th + kTwoPiF : th;
        it = min((int)(th * g.inv_dth), n_t - 1);
    } else {
        // angle from the tile's first boundary, wrapped to [-pi, pi): a point just below
        // theta = 2 pi belongs to a tile starting at 0 (the tile spans <= pi/2)
        float rel = th - (float)t.t0 * g.dth;
        rel = rel < -0.5f * kTwoPiF ? rel + kTwoPiF : (rel >= 0.5f * kTwoPiF ? rel - kTwoPiF : rel);
        it = t.t0 + min(max((int)floorf(rel * g.inv_dth), 0), t.t1 - t.t0 - 1);
    }
    int ih = min(max((int)floorf((z - g.h0) * g.inv_dh), t.s0), t.s1 - 1);

    bool inward = u < 0.f;
    const float d2 = rr.b.w, utan = rr.a.w, dr = g.dr;
    const float inv_a = radial ? 1.f / fmaf(ex, ex, ey * ey) : 0.f;
    auto next_r = [&](int ir_, bool inw, float ucur) -> float {
        if (!radial) return kInf;
        int k;
        float sgn;
        if (inw && ir_ >= kstar) { k = ir_; sgn = -1.f; }
        else { k = ir_ + 1; sgn = 1.f; }
        if (k >= n_r) return kInf;
        float rk = k * dr;
        float q = (k == kstar) ? utan : fsqrt_fast(fmaxf(fmaf(rk, rk, -d2), 0.f) * inv_a);
        return fmaxf(sgn * q, ucur);
    };
    auto next_t = [&](int it_, float ucur) -> float {
        if (n_t == 1 || !radial) return kInf;
        int k;
        if (ccw) {
            k = it_ + 1;
            if (!t.full_circle && k >= t.t1) return kInf;
            k = (k == n_t) ? 0 : k;
        } else {
            if (!t.full_circle && it_ <= t.t0) return kInf;
            k = it_;
        }
        float2 cs = trig[k];
        float nd = cs.x * ey - cs.y * ex;
        if (sense * nd <= 0.f) return kInf;
        float no = cs.x * py - cs.y * px;
        return fmaxf(__fdividef(-no, nd), ucur);
    };
    auto next_h = [&](int ih_, float ucur) -> float {
        if (ez > 0.f) return (ih_ + 1 < t.s1) ? fmaxf(fmaf((float)(ih_ + 1), c1, c0), ucur) : kInf;
        if (ez < 0.f) return (ih_ > t.s0) ? fmaxf(fmaf((float)ih_, c1, c0), ucur) : kInf;
        return kInf;
    };

    float ur = next_r(ir, inward, u);
    float ut = next_t(it, u);
    float uh = next_h(ih, u);
    const int tw = t.t1 - t.t0;
    const int tstep = n_r, hstep = tw * n_r;
    int idx = ((ih - t.s0) * tw + (it - t.t0)) * n_r + ir;
    for (int step = 0; step < g.max_steps; ++step) {
        float un = fminf(fminf(ur, ut), uh);
        float ue = fminf(un, ub);
        op(idx, ue - u);
        if (un >= ub) break;
        u = un;
        if (un == ur) {
            if (inward && ir >= kstar) { ir -= 1; idx -= 1; }
            else { inward = false; ir += 1; idx += 1; }
            ur = next_r(ir, inward, u);
        } else if (un == ut) {
            if (ccw) {
                if (it + 1 == n_t) { it = 0; idx -= (n_t - 1) * tstep; }
                else { it += 1; idx += tstep; }
            } else {
                if (it == 0) { it = n_t - 1; idx += (n_t - 1) * tstep; }
                else { it -= 1; idx -= tstep; }
            }
            ut = next_t(it, u);
        } else {
            if (ez > 0.f) { ih += 1; idx += hstep; }
            else { ih -= 1; idx -= hstep; }
            uh = next_h(ih, u);
        }
    }
    return true;
}

}  // namespace cylct
