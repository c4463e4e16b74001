// Exact ray traversal of the cylindrical grid (device code).
//
// t_jl of Sec. 2.2 (Eq. 6) is the length of ray j inside voxel l.  A voxel of the grid of
// Eq. 2 is bounded by two radial shells, two azimuthal wedge half-planes and two axial
// slab planes, so a ray's row of the system matrix is the list of pieces between
// consecutive crossings of those three families.  A ray walks them incrementally: it
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
// A walk may start anywhere inside the clipped interval (the kernels cut a ray into
// pieces walked by different threads): the start voxel comes from the start point, the
// next crossing of each family from the formulas above.
//
// Robustness: every crossing is clamped to be >= the current position and every index
// change is a single step, so rounding near a boundary only creates a zero-length piece.
// Indices never leave the grid (its exits are the clip, not crossings), and a walk stops
// after max_steps pieces.
#pragma once

#include "cylct_internal.h"

namespace cylct {

constexpr float kInf = 3.0e38f;
constexpr float kTwoPiF = 6.283185307179586f;

// Weight-map elements as FP32 (Sec. 2.2 weighted back-projection): FP32, FP16, BF16, or
// the byte values of a U8 class map.
__device__ __forceinline__ float weight_f32(float v) { return v; }
__device__ __forceinline__ float weight_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float weight_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float weight_f32(uint8_t v) { return (float)v; }

// FP32 ray record, computed once per plan and pose in FP64 (k_rays).
//   a = (P*x, P*y, uref, utan)  uref: u of slab plane kref (or 0 for a ray with e_z = 0)
//                               utan: |u| of shell boundary kstar
//   b = (e_x, e_y, e_z, d^2)
//   c = (u_in, u_out, L, packed) L: chord in the grid cylinder (row sum of Eq. 7);
//                               u_in > u_out marks a ray that misses the grid;
//                               packed = kstar | kref << 16, kstar = 0xffff for a ray
//                               parallel to the axis; kref: the slab plane nearest the
//                               chord's midpoint (the slab holding the ray if e_z = 0).
// Slab crossings are uref + (k - kref) dh / e_z: measured from a plane next to the chord,
// they keep FP32 accuracy for rays almost parallel to the planes, where z* + u e_z
// would cancel.
struct RayRec {
    float4 a, b, c;
};

constexpr int kNoShell = 0xffff;

__device__ __forceinline__ int ray_kstar(const RayRec &rr)
{
    const int k = __float_as_int(rr.c.w) & 0xffff;
    return k == kNoShell ? -1 : k;
}

__device__ __forceinline__ int ray_kref(const RayRec &rr)
{
    return (int)((unsigned)__float_as_int(rr.c.w) >> 16);
}

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
    int ks = kNoShell;
    float utan = 0.f;
    if (radial) {
        ks = (int)floor(sqrt(d2) / g.dr_d) + 1;
        if (ks < g.n_r) {
            double rk = ks * g.dr_d;
            utan = (float)sqrt(fmax(rk * rk - d2, 0.0) * inv_a);
        }
    }
    const double zs = Sz + sstar * ez;          // z at the closest approach
    const double dh = g.height / g.n_h;
    int kref;
    double uref = 0.0;
    if (ez != 0.0) {
        const double zm = zs + 0.5 * (s_lo + s_hi - 2.0 * sstar) * ez;
        kref = (int)fmin(fmax(floor((zm + half) / dh + 0.5), 0.0), (double)g.n_h);
        uref = (-half + kref * dh - zs) / ez;
    } else {
        kref = (int)fmin(fmax(floor((zs + half) / dh), 0.0), (double)(g.n_h - 1));
    }
    rr.a = make_float4((float)(Sx + sstar * ex), (float)(Sy + sstar * ey), (float)uref, utan);
    rr.b = make_float4((float)ex, (float)ey, (float)ez, (float)d2);
    rr.c = make_float4((float)(s_lo - sstar), (float)(s_hi - sstar), (float)(s_hi - s_lo),
                       __int_as_float(ks | (kref << 16)));
    return rr;
}

// State of one ray walking the grid.  Each family keeps its next crossing and what it
// needs to find the one after:
//   shells: ks, a signed count of the next boundary: -k for boundary k crossed inward
//           (ir: k -> k-1), +k crossed outward (ir: k-1 -> k).  Inward the count runs
//           -k_0, -(k_0-1), .., -kstar, then turns to +kstar, +(kstar+1), ..; boundary k
//           sits at u = sign(ks) sqrt(A k^2 + B), A = dr^2 / a, B = -d^2 / a (utan for
//           kstar, whose crossing can be near-tangent); the radius R (ks = N_r) is the
//           clip, never a crossing.
//   wedges: kt, the next boundary, and dt = +-1 the sense theta moves in.  P* and e are
//           stored multiplied by dt, so boundary k is crossed on its own half-plane iff
//           n_k . e' > 0, at u = -(n_k . P*') / (n_k . e').
//   slabs:  kh, the next slab plane minus kref, as a float: u = uref + kh c1,
//           c1 = dh / e_z; planes 0 and N_h are the clip.
// The voxel index changes by -1 / +1 at a shell, +-N_r (wrapping at wedge 0) at a wedge
// and +-N_theta N_r at a slab.
struct Walker {
    float px, py, ex, ey;     // P* and e in the x'y' plane, times dt
    float A, B, utan;
    float kstar_f, nr_f;      // kstar and N_r as floats
    float c1, uref;           // uref = +inf for a ray with e_z = 0
    float kh_lo, kh_hi;       // valid planes: kh_lo < kh < kh_hi
    float hsign;              // +-1: the slab direction (0 with e_z = 0)
    float u, ub, ur, ut, uh, ks, kh;
    int idx, kt, dt, nt, dtn, dtw, hstep, left;

    __device__ __forceinline__ float shell_u(float k) const
    {
        const float q2 = fmaxf(fmaf(A * k, k, B), 0.f);
        const float q = fabsf(k) == kstar_f ? utan : q2 * rsqrtf(fmaxf(q2, 1e-30f));
        const float us = copysignf(q, k);
        return k >= nr_f ? kInf : fmaxf(us, u);
    }
    __device__ __forceinline__ float wedge_u(const float2 *__restrict__ trig, int k) const
    {
        const float2 cs = trig[k];
        const float nd = cs.x * ey - cs.y * ex, no = cs.x * py - cs.y * px;
        const float uw = fmaxf(__fdividef(-no, nd), u);
        return nd > 0.f ? uw : kInf;
    }
    __device__ __forceinline__ float slab_u(float k) const
    {
        const float uz = fmaxf(fmaf(k, c1, uref), u);
        return (k > kh_lo && k < kh_hi) ? uz : kInf;
    }

    // Start at ua on ray rr; the walk ends at ub.
    __device__ __forceinline__ void init(const GridDev &g, const float2 *__restrict__ trig,
                                         const RayRec &rr, float ua, float ub_)
    {
        const float ez = rr.b.z;
        const int kstar = ray_kstar(rr), kref = ray_kref(rr);
        const bool radial = kstar >= 0;
        px = rr.a.x;
        py = rr.a.y;
        ex = rr.b.x;
        ey = rr.b.y;
        const float inv_a = radial ? 1.f / fmaf(ex, ex, ey * ey) : 0.f;
        A = g.dr * g.dr * inv_a;
        B = -rr.b.w * inv_a;
        utan = rr.a.w;
        kstar_f = (float)kstar;
        nr_f = (float)g.n_r;
        u = ua;
        ub = ub_;
        left = g.max_steps;
        nt = g.n_t;
        // start voxel
        const float x = fmaf(u, ex, px), y = fmaf(u, ey, py);
        const int ir = min((int)(sqrtf(fmaf(x, x, y * y)) * g.inv_dr), g.n_r - 1);
        float th = atan2f(y, x);
        th = th < 0.f ? th + kTwoPiF : th;
        const int it = min((int)(th * g.inv_dth), g.n_t - 1);
        const int ih = ez != 0.f ? min(max(kref + (int)floorf((u - rr.a.z) * ez * g.inv_dh), 0), g.n_h - 1)
                                 : kref;
        idx = (ih * g.n_t + it) * g.n_r + ir;
        // shells
        if (!radial) ks = nr_f;
        else if (u < 0.f && ir >= kstar) ks = -(float)ir;
        else ks = (float)(ir + 1);
        // wedges: counter-clockwise the far edge of wedge it is next, else its own edge
        const bool ccw = (px * ey - py * ex) >= 0.f;
        dt = ccw ? 1 : -1;
        const float s = ccw ? 1.f : -1.f;
        px *= s;
        py *= s;
        ex *= s;
        ey *= s;
        kt = ccw ? (it + 1 == g.n_t ? 0 : it + 1) : it;
        dtn = dt * g.n_r;
        dtw = -dt * (g.n_t - 1) * g.n_r;
        const bool wedges = radial && g.n_t > 1;
        // slabs
        hsign = ez > 0.f ? 1.f : (ez < 0.f ? -1.f : 0.f);
        c1 = ez != 0.f ? g.dh / ez : 0.f;
        uref = ez != 0.f ? rr.a.z : kInf;
        kh = (float)((ez > 0.f ? ih + 1 : ih) - kref);
        kh_lo = (float)(-kref);
        kh_hi = (float)(g.n_h - kref);
        hstep = (ez > 0.f ? 1 : -1) * g.n_t * g.n_r;
        ur = shell_u(ks);
        if (!wedges) kt = 0;
        ut = wedges ? wedge_u(trig, kt) : kInf;
        uh = slab_u(kh);
    }

    // One piece: calls op(idx, length); returns false once the ray has reached ub (or
    // after max_steps pieces).  Branch-free: the next crossing of every family is
    // evaluated and the one of the family that moved is kept.
    template <class Op>
    __device__ __forceinline__ bool step(const GridDev &g, const float2 *__restrict__ trig, Op &op)
    {
        const float un = fminf(fminf(ur, ut), uh);
        op(idx, fminf(un, ub) - u);
        if (un >= ub || --left <= 0) return false;
        u = un;
        const bool isr = un == ur;
        const bool ist = !isr && un == ut;
        const bool ish = !isr && !ist;
        // index change of the family that moved
        const int d_r = ks < 0.f ? -1 : 1;
        const int d_t = kt == 0 ? dtw : dtn;
        idx += isr ? d_r : (ist ? d_t : hstep);
        // advance that family
        const float ks2 = ks == -kstar_f ? kstar_f : ks + 1.f;
        int kt2 = kt + dt;
        kt2 = kt2 == nt ? 0 : (kt2 < 0 ? nt - 1 : kt2);
        ks = isr ? ks2 : ks;
        kt = ist ? kt2 : kt;
        kh = ish ? kh + hsign : kh;
        // its next crossing
        const float urn = shell_u(ks);
        const float utn = wedge_u(trig, kt);
        const float uhn = slab_u(kh);
        ur = isr ? urn : ur;
        ut = ist ? utn : ut;
        uh = ish ? uhn : uh;
        return true;
    }
};

}  // namespace cylct
