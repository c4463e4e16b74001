// Host geometry (FP64): validation, the alignment of Eq. 1, per-view geometry tables and
// the grid constants with the wedge table.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

namespace cylct {

// Rotation of the alignment of Eq. 1: R = O^T with O = Rz(alpha) Rx(beta) Rz(gamma),
// written out in closed form.
void alignment_matrix(const cyl_pose &ps, double R[3][3])
{
    const double ca = cos(ps.alpha), sa = sin(ps.alpha);
    const double cb = cos(ps.beta), sb = sin(ps.beta);
    const double cg = cos(ps.gamma), sg = sin(ps.gamma);
    const double O[3][3] = {
        {ca * cg - sa * cb * sg, -ca * sg - sa * cb * cg, sa * sb},
        {sa * cg + ca * cb * sg, -sa * sg + ca * cb * cg, -ca * sb},
        {sb * sg, sb * cg, cb},
    };
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = O[j][i];
}

int validate_geom(const cyl_geom *geom)
{
    if (!geom) return set_error(CYL_EINVAL, "null geometry");
    if (geom->n_proj < 1 || geom->det_w < 1 || geom->det_h < 1)
        return set_error(CYL_EINVAL, "projections and detector size must be >= 1");
    if ((int64_t)geom->det_w * geom->det_h >= (int64_t)1 << 30)
        return set_error(CYL_EINVAL, "detector must have fewer than 2^30 pixels");
    if (geom->frames_mm) {
        for (int64_t k = 0; k < 12 * (int64_t)geom->n_proj; ++k)
            if (!std::isfinite(geom->frames_mm[k])) return set_error(CYL_EINVAL, "non-finite frame");
        for (int p = 0; p < geom->n_proj; ++p) {
            const double *f = geom->frames_mm + 12 * (int64_t)p;
            const double du = std::sqrt(f[6] * f[6] + f[7] * f[7] + f[8] * f[8]);
            const double dv = std::sqrt(f[9] * f[9] + f[10] * f[10] + f[11] * f[11]);
            if (!(du > 0.0) || !(dv > 0.0)) return set_error(CYL_EINVAL, "zero pixel step in a frame");
            // the detector plane must not contain the source
            const double n[3] = {f[7] * f[11] - f[8] * f[10], f[8] * f[9] - f[6] * f[11], f[6] * f[10] - f[7] * f[9]};
            const double h = n[0] * (f[3] - f[0]) + n[1] * (f[4] - f[1]) + n[2] * (f[5] - f[2]);
            if (!(std::fabs(h) > 0.0)) return set_error(CYL_EINVAL, "a frame's source lies in its detector plane");
        }
        return CYL_OK;
    }
    if (!(geom->sod_mm > 0.0) || !(geom->sdd_mm > geom->sod_mm) || !std::isfinite(geom->sdd_mm))
        return set_error(CYL_EINVAL, "need 0 < SOD < SDD");
    if (!(geom->pitch_u_mm > 0.0) || !(geom->pitch_v_mm > 0.0) ||
        !std::isfinite(geom->pitch_u_mm) || !std::isfinite(geom->pitch_v_mm))
        return set_error(CYL_EINVAL, "pixel pitch must be finite and > 0");
    if (!std::isfinite(geom->off_u_mm) || !std::isfinite(geom->off_v_mm))
        return set_error(CYL_EINVAL, "detector offset must be finite");
    if (!geom->angles_rad) return set_error(CYL_EINVAL, "angles_rad is null");
    for (int p = 0; p < geom->n_proj; ++p)
        if (!std::isfinite(geom->angles_rad[p])) return set_error(CYL_EINVAL, "non-finite angle");
    return CYL_OK;
}

int validate_scan(const cyl_grid *grid, const cyl_geom *geom, const cyl_pose *pose)
{
    if (!grid || !geom || !pose) return set_error(CYL_EINVAL, "null grid, geometry or pose");
    if (grid->n_h < 1 || grid->n_theta < 1 || grid->n_r < 1)
        return set_error(CYL_EINVAL, "grid divisions must be >= 1");
    if (grid->n_r > 65534 || grid->n_h > 65535)
        return set_error(CYL_EINVAL, "n_r must be <= 65534 and n_h <= 65535");
    if (grid->n_theta > CYL_MAX_N_THETA)
        return set_error(CYL_EINVAL, "n_theta must be <= 6144 (wedge table in shared memory)");
    if ((int64_t)grid->n_h * grid->n_theta * grid->n_r >= (int64_t)1 << 31)
        return set_error(CYL_EINVAL, "grid must have fewer than 2^31 voxels");
    if (!(grid->radius_mm > 0.0) || !(grid->height_mm > 0.0) || !std::isfinite(grid->radius_mm) ||
        !std::isfinite(grid->height_mm))
        return set_error(CYL_EINVAL, "grid radius and height must be finite and > 0");
    int rc = validate_geom(geom);
    if (rc) return rc;
    const double pv[6] = {pose->alpha, pose->beta, pose->gamma, pose->tx, pose->ty, pose->tz};
    for (double v : pv)
        if (!std::isfinite(v)) return set_error(CYL_EINVAL, "non-finite pose");
    // the grid cylinder, wherever the pose puts it, must not reach any source
    const double sphere = std::sqrt(grid->radius_mm * grid->radius_mm +
                                    0.25 * grid->height_mm * grid->height_mm);
    if (geom->frames_mm) {
        for (int p = 0; p < geom->n_proj; ++p) {
            const double *f = geom->frames_mm + 12 * (int64_t)p;
            const double sx = f[0] - pose->tx, sy = f[1] - pose->ty, sz = f[2] - pose->tz;
            if (std::sqrt(sx * sx + sy * sy + sz * sz) <= sphere)
                return set_error(CYL_EINVAL, "the grid cylinder reaches a frame's source");
        }
        return CYL_OK;
    }
    const double reach = sphere + std::sqrt(pose->tx * pose->tx + pose->ty * pose->ty + pose->tz * pose->tz);
    if (reach >= geom->sod_mm) return set_error(CYL_EINVAL, "the grid cylinder reaches the source");
    return CYL_OK;
}

void build_grid(const cyl_grid &grid, const cyl_geom &geom, GridDev &g, std::vector<float2> &trig)
{
    trig.resize(grid.n_theta);
    for (int k = 0; k < grid.n_theta; ++k) {
        const double th = 2.0 * M_PI * k / grid.n_theta;
        trig[k] = make_float2((float)cos(th), (float)sin(th));
    }
    g.n_h = grid.n_h;
    g.n_t = grid.n_theta;
    g.n_r = grid.n_r;
    g.det_w = geom.det_w;
    g.det_h = geom.det_h;
    g.max_steps = 2 * grid.n_r + grid.n_theta + grid.n_h + 8;
    g.radius = grid.radius_mm;
    g.height = grid.height_mm;
    g.dr_d = grid.radius_mm / grid.n_r;
    g.dr = (float)g.dr_d;
    g.inv_dr = (float)(grid.n_r / grid.radius_mm);
    g.dth = (float)(2.0 * M_PI / grid.n_theta);
    g.inv_dth = (float)(grid.n_theta / (2.0 * M_PI));
    g.dh = (float)(grid.height_mm / grid.n_h);
    g.inv_dh = (float)(grid.n_h / grid.height_mm);
    g.h0 = (float)(-0.5 * grid.height_mm);
    // Floor of Eq. 7's row and column sums: far below any voxel size, well above the
    // FP32 walk's position error, so a grazed ray or voxel moves by (chord / eps)^2 of its
    // plain update
    g.eps = (float)ldexp(grid.radius_mm, -16);
}

void build_views(const cyl_geom &geom, const cyl_pose &pose, std::vector<ProjGeom> &geo)
{
    double R[3][3];
    alignment_matrix(pose, R);
    const double T[3] = {pose.tx, pose.ty, pose.tz};
    const int W = geom.det_w, H = geom.det_h;
    geo.resize(geom.n_proj);
    const double xd = geom.sdd_mm - geom.sod_mm;
    const double u0 = -0.5 * (W - 1) * geom.pitch_u_mm + geom.off_u_mm;
    const double v0 = -0.5 * (H - 1) * geom.pitch_v_mm + geom.off_v_mm;
    for (int p = 0; p < geom.n_proj; ++p) {
        if (geom.frames_mm) {           // general trajectory: stage coordinates, no turn
            const double *f = geom.frames_mm + 12 * (int64_t)p;
            auto to_obj = [&](const double *st0, bool point, double out[3]) {
                double st[3] = {st0[0], st0[1], st0[2]};
                if (point)
                    for (int i = 0; i < 3; ++i) st[i] -= T[i];
                for (int i = 0; i < 3; ++i) out[i] = R[i][0] * st[0] + R[i][1] * st[1] + R[i][2] * st[2];
            };
            to_obj(f, true, geo[p].S);
            to_obj(f + 3, true, geo[p].D0);
            to_obj(f + 6, false, geo[p].du);
            to_obj(f + 9, false, geo[p].dv);
            continue;
        }
        const double c = cos(geom.angles_rad[p]), s = sin(geom.angles_rad[p]);
        // lab -> stage: Rz(-phi); then X' = R (X - T)
        auto to_obj = [&](const double lab[3], bool point, double out[3]) {
            double st[3] = {c * lab[0] + s * lab[1], -s * lab[0] + c * lab[1], lab[2]};
            if (point)
                for (int i = 0; i < 3; ++i) st[i] -= T[i];
            for (int i = 0; i < 3; ++i) out[i] = R[i][0] * st[0] + R[i][1] * st[1] + R[i][2] * st[2];
        };
        const double src[3] = {-geom.sod_mm, 0.0, 0.0};
        const double d00[3] = {xd, u0, v0};
        const double du[3] = {0.0, geom.pitch_u_mm, 0.0};
        const double dv[3] = {0.0, 0.0, geom.pitch_v_mm};
        to_obj(src, true, geo[p].S);
        to_obj(d00, true, geo[p].D0);
        to_obj(du, false, geo[p].du);
        to_obj(dv, false, geo[p].dv);
    }
}

}  // namespace cylct

namespace cylct {

double hit_fraction_bound(const cyl_grid &grid, const cyl_geom &geom, const std::vector<ProjGeom> &geo)
{
    constexpr int kRim = 64;
    const double W = geom.det_w, H = geom.det_h;
    double covered = 0.0;
    for (const ProjGeom &v : geo) {
        // pixel coordinates (a, b) of an object point: D0 + a du + b dv on the line from S
        const double n[3] = {v.du[1] * v.dv[2] - v.du[2] * v.dv[1], v.du[2] * v.dv[0] - v.du[0] * v.dv[2],
                             v.du[0] * v.dv[1] - v.du[1] * v.dv[0]};
        double e1[3], e2[3];
        {
            const double t1[3] = {v.dv[1] * n[2] - v.dv[2] * n[1], v.dv[2] * n[0] - v.dv[0] * n[2],
                                  v.dv[0] * n[1] - v.dv[1] * n[0]};
            const double t2[3] = {n[1] * v.du[2] - n[2] * v.du[1], n[2] * v.du[0] - n[0] * v.du[2],
                                  n[0] * v.du[1] - n[1] * v.du[0]};
            const double q1 = t1[0] * v.du[0] + t1[1] * v.du[1] + t1[2] * v.du[2];
            const double q2 = t2[0] * v.dv[0] + t2[1] * v.dv[1] + t2[2] * v.dv[2];
            for (int k = 0; k < 3; ++k) {
                e1[k] = t1[k] / q1;
                e2[k] = t2[k] / q2;
            }
        }
        const double c0 = n[0] * (v.D0[0] - v.S[0]) + n[1] * (v.D0[1] - v.S[1]) + n[2] * (v.D0[2] - v.S[2]);
        double a_lo = 1e300, a_hi = -1e300, b_lo = 1e300, b_hi = -1e300;
        bool ok = true;
        for (int side = 0; side < 2 && ok; ++side)
            for (int k = 0; k < kRim; ++k) {
                // rim points of a slightly larger polygon that contains the circle
                const double th = 2.0 * M_PI * k / kRim, rr = grid.radius_mm / cos(M_PI / kRim);
                const double X[3] = {rr * cos(th), rr * sin(th), (side ? 0.5 : -0.5) * grid.height_mm};
                const double Y[3] = {X[0] - v.S[0], X[1] - v.S[1], X[2] - v.S[2]};
                const double nY = n[0] * Y[0] + n[1] * Y[1] + n[2] * Y[2];
                const double t = c0 / nY;
                if (!(t > 0.0) || !std::isfinite(t)) {   // the point is not in front of the source
                    ok = false;
                    break;
                }
                const double P[3] = {v.S[0] + t * Y[0] - v.D0[0], v.S[1] + t * Y[1] - v.D0[1],
                                     v.S[2] + t * Y[2] - v.D0[2]};
                const double a = e1[0] * P[0] + e1[1] * P[1] + e1[2] * P[2];
                const double b = e2[0] * P[0] + e2[1] * P[1] + e2[2] * P[2];
                a_lo = std::min(a_lo, a);
                a_hi = std::max(a_hi, a);
                b_lo = std::min(b_lo, b);
                b_hi = std::max(b_hi, b);
            }
        if (!ok) return 1.0;
        // pixel centres a in [0, W - 1]; a box [a_lo, a_hi] holds at most this many
        const double wa = std::max(0.0, std::min(W - 1.0, std::floor(a_hi)) - std::max(0.0, std::ceil(a_lo)) + 1.0);
        const double wb = std::max(0.0, std::min(H - 1.0, std::floor(b_hi)) - std::max(0.0, std::ceil(b_lo)) + 1.0);
        covered += wa * wb;
    }
    return covered / (W * H * (double)geo.size());
}

}  // namespace cylct
