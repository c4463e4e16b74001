// Exact ray traversal of the cylindrical grid (device code).
//
// t_jl of Sec. 2.2 (Eq. 5) is the length of ray j inside voxel l.  A voxel of the grid of
// Eq. 2 is bounded by two radial shells, two azimuthal wedge half-planes and two axial
// slab planes, so a ray's row of the system matrix is the list of pieces between
// consecutive crossings of those three families.  Instead of collecting and sorting
// crossings, each ray walks them incrementally: it keeps the next crossing of each
// family and always advances the nearest one, so the voxel index changes by one step of
// one family at a time.
//
// Parametrisation.  u is the distance (mm) along the ray from its closest approach to
// the z' axis.  With a = e_x^2 + e_y^2 and d the axis distance,
//     r(u)^2 = a u^2 + d^2,   so shell k is crossed at u = -+sqrt((r_k^2 - d^2) / a);
//     theta(u) is monotone (sense = sign of (P* x e)_z), wedge boundary k is crossed at
//     u = -(n_k . P*) / (n_k . e), n_k = (-sin theta_k, cos theta_k), and only if the
//     crossing is on the theta_k half-plane, i.e. sense * (n_k . e) > 0;
//     h(u) = z* + u e_z, slab k is crossed at u = (h_k - z*) / e_z.
// Measuring u from the closest approach keeps every position small (|u| <= R-ish), so
// the walk runs in FP32; the ray set-up (clip to the grid cylinder, closest approach,
// axis distance, row sum) runs in FP64, and so does the one shell crossing that can be
// near-tangent (the innermost shell boundary the ray reaches).
//
// Robustness: every crossing is clamped to be >= the current position and every index
// change is a single step, so rounding near a boundary only creates a zero-length piece.
// Indices never leave the grid (the exit is the FP64 clip, not a crossing), and the walk
// stops after max_steps pieces.
#pragma once

#include "cylct_internal.h"

namespace cylct {

constexpr float kInf = 3.0e38f;
constexpr float kTwoPiF = 6.283185307179586f;

struct Ray {
    float px, py, pz;   // closest approach point P* (FP32)
    float ex, ey, ez;   // unit direction
    float inv_a;        // 1 / (e_x^2 + e_y^2)
    float d2;           // squared axis distance of the line
    float u_in, u_out;  // clipped interval, mm from P*
    float utan;         // |u| of shell boundary kstar (FP64-derived)
    float L;            // chord length = row sum of Eq. 6
    int kstar;          // first shell boundary above the axis distance
    bool hit;
    bool radial;        // false: ray parallel to the axis (no shell / wedge crossings)
};

__device__ __forceinline__ float fsqrt_fast(float x)
{
    return x > 0.f ? x * rsqrtf(x) : 0.f;
}

// FP64 set-up of ray (p, iu, iv): clip to {r <= R, |h| <= H/2} and the source-pixel
// segment, closest approach, and the near-tangent shell crossing.
__device__ __forceinline__ Ray setup_ray(const GridDev &g, const ProjGeom &pg, int iu, int iv)
{
    Ray ry;
    ry.hit = false;
    ry.radial = true;
    double Sx = pg.S[0], Sy = pg.S[1], Sz = pg.S[2];
    double Dx = pg.D0[0] + iu * pg.du[0] + iv * pg.dv[0];
    double Dy = pg.D0[1] + iu * pg.du[1] + iv * pg.dv[1];
    double Dz = pg.D0[2] + iu * pg.du[2] + iv * pg.dv[2];
    double dx = Dx - Sx, dy = Dy - Sy, dz = Dz - Sz;
    double len = sqrt(dx * dx + dy * dy + dz * dz);
    double inv_len = 1.0 / len;
    double ex = dx * inv_len, ey = dy * inv_len, ez = dz * inv_len;
    double a = ex * ex + ey * ey;
    double R = g.radius, half = 0.5 * g.height;
    double s_lo, s_hi, sstar, d2;
    if (a > 1e-18) {
        double m = Sx * ey - Sy * ex;            // (S x e)_z: a * d^2 = m^2
        d2 = m * m / a;
        if (d2 >= R * R) return ry;
        sstar = -(Sx * ex + Sy * ey) / a;
        double hR = sqrt((R * R - d2) / a);
        s_lo = fmax(sstar - hR, 0.0);
        s_hi = fmin(sstar + hR, len);
    } else {                                      // parallel to the axis
        d2 = Sx * Sx + Sy * Sy;
        if (d2 > R * R) return ry;
        ry.radial = false;
        sstar = 0.0;
        s_lo = 0.0;
        s_hi = len;
    }
    if (ez != 0.0) {
        double s1 = (-half - Sz) / ez, s2 = (half - Sz) / ez;
        s_lo = fmax(s_lo, fmin(s1, s2));
        s_hi = fmin(s_hi, fmax(s1, s2));
    } else if (Sz < -half || Sz > half) {
        return ry;
    }
    if (!(s_hi > s_lo)) return ry;
    ry.hit = true;
    ry.px = (float)(Sx + sstar * ex);
    ry.py = (float)(Sy + sstar * ey);
    ry.pz = (float)(Sz + sstar * ez);
    ry.ex = (float)ex;
    ry.ey = (float)ey;
    ry.ez = (float)ez;
    ry.inv_a = ry.radial ? (float)(1.0 / a) : 0.f;
    ry.d2 = (float)d2;
    ry.u_in = (float)(s_lo - sstar);
    ry.u_out = (float)(s_hi - sstar);
    ry.L = (float)(s_hi - s_lo);
    double d = sqrt(d2);
    int ks = (int)floor(d / g.dr_d) + 1;
    ry.kstar = ks;
    ry.utan = 0.f;
    if (ry.radial && ks < g.n_r) {
        double rk = ks * g.dr_d;
        ry.utan = (float)sqrt(fmax(rk * rk - d2, 0.0) / a);
    }
    return ry;
}

// Walk the pieces of a hit ray, calling op(voxel, length) for each in order along the
// ray (zero-length pieces included).
template <class Op>
__device__ __forceinline__ void walk_ray(const GridDev &g, const float2 *__restrict__ trig,
                                         const Ray &ry, Op &op)
{
    const int n_r = g.n_r, n_t = g.n_t, n_h = g.n_h;
    float u = ry.u_in;
    const float u_out = ry.u_out;
    // entry indices from the entry point
    float x = fmaf(u, ry.ex, ry.px), y = fmaf(u, ry.ey, ry.py), z = fmaf(u, ry.ez, ry.pz);
    int ir = min((int)(sqrtf(fmaf(x, x, y * y)) * g.inv_dr), n_r - 1);
    float th = atan2f(y, x);
    th = th < 0.f ? th + kTwoPiF : th;
    int it = min((int)(th * g.inv_dth), n_t - 1);
    int ih = max(min((int)floorf((z - g.h0) * g.inv_dh), n_h - 1), 0);

    // radial family
    bool inward = u < 0.f;
    const float d2 = ry.d2, inv_a = ry.inv_a, utan = ry.utan, dr = g.dr;
    const int kstar = ry.kstar;
    auto next_r = [&](int ir_, bool inw, float ucur) -> float {
        if (!ry.radial) return kInf;
        int k;
        float sgn;
        if (inw && ir_ >= kstar) { k = ir_; sgn = -1.f; }
        else { k = ir_ + 1; sgn = 1.f; }
        if (k >= n_r) return kInf;
        float rk = k * dr;
        float q = (k == kstar) ? utan : fsqrt_fast(fmaxf(fmaf(rk, rk, -d2), 0.f) * inv_a);
        return fmaxf(sgn * q, ucur);
    };
    // azimuthal family
    const float px = ry.px, py = ry.py, ex = ry.ex, ey = ry.ey;
    const float sense = (px * ey - py * ex) >= 0.f ? 1.f : -1.f;
    const bool ccw = sense > 0.f;
    auto next_t = [&](int it_, float ucur) -> float {
        if (n_t == 1 || !ry.radial) return kInf;
        int k = ccw ? it_ + 1 : it_;
        k = (k == n_t) ? 0 : k;
        float2 cs = trig[k];
        float nd = cs.x * ey - cs.y * ex;
        if (sense * nd <= 0.f) return kInf;
        float no = cs.x * py - cs.y * px;
        return fmaxf(__fdividef(-no, nd), ucur);
    };
    // axial family
    const float ez = ry.ez;
    const float inv_ez = ez != 0.f ? 1.f / ez : 0.f;
    const float c0 = (g.h0 - ry.pz) * inv_ez, c1 = g.dh * inv_ez;
    auto next_h = [&](int ih_, float ucur) -> float {
        if (ez > 0.f) return (ih_ + 1 < n_h) ? fmaxf(fmaf((float)(ih_ + 1), c1, c0), ucur) : kInf;
        if (ez < 0.f) return (ih_ > 0) ? fmaxf(fmaf((float)ih_, c1, c0), ucur) : kInf;
        return kInf;
    };

    float ur = next_r(ir, inward, u);
    float ut = next_t(it, u);
    float uh = next_h(ih, u);
    int idx = (ih * n_t + it) * n_r + ir;
    const int rstep = 1, tstep = n_r, hstep = n_t * n_r;
    for (int step = 0; step < g.max_steps; ++step) {
        float un = fminf(fminf(ur, ut), uh);
        float ue = fminf(un, u_out);
        op(idx, ue - u);
        if (un >= u_out) break;
        u = un;
        if (un == ur) {
            if (inward && ir >= kstar) { ir -= 1; idx -= rstep; }
            else { inward = false; ir += 1; idx += rstep; }
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
}

}  // namespace cylct
