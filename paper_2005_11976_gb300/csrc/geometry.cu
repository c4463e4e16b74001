// Host geometry (FP64): validation, the alignment of Eq. 1, per-view ray tables, the
// wedge table, the volume tiling and each tile's candidate pixel box per view.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

namespace cylct {

// Rotation of the alignment of Eq. 1: R = O^T with O = Rz(alpha) Rx(beta) Rz(gamma),
// written out in closed form.
static void alignment_matrix(const cyl_pose &ps, double R[3][3])
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

int validate_scan(const cyl_grid *grid, const cyl_geom *geom, const cyl_pose *pose)
{
    if (!grid || !geom || !pose) return set_error(CYL_EINVAL, "null grid, geometry or pose");
    if (grid->n_h < 1 || grid->n_theta < 1 || grid->n_r < 1)
        return set_error(CYL_EINVAL, "grid divisions must be >= 1");
    if ((int64_t)grid->n_h * grid->n_theta * grid->n_r >= (int64_t)1 << 31)
        return set_error(CYL_EINVAL, "grid must have fewer than 2^31 voxels");
    if (!(grid->radius_mm > 0.0) || !(grid->height_mm > 0.0) || !std::isfinite(grid->radius_mm) ||
        !std::isfinite(grid->height_mm))
        return set_error(CYL_EINVAL, "grid radius and height must be finite and > 0");
    if (!(geom->sod_mm > 0.0) || !(geom->sdd_mm > geom->sod_mm) || !std::isfinite(geom->sdd_mm))
        return set_error(CYL_EINVAL, "need 0 < SOD < SDD");
    if (geom->n_proj < 1 || geom->det_w < 1 || geom->det_h < 1)
        return set_error(CYL_EINVAL, "projections and detector size must be >= 1");
    if ((int64_t)geom->det_w * geom->det_h >= (int64_t)1 << 30)
        return set_error(CYL_EINVAL, "detector must have fewer than 2^30 pixels");
    if (!(geom->pitch_u_mm > 0.0) || !(geom->pitch_v_mm > 0.0) ||
        !std::isfinite(geom->pitch_u_mm) || !std::isfinite(geom->pitch_v_mm))
        return set_error(CYL_EINVAL, "pixel pitch must be finite and > 0");
    if (!std::isfinite(geom->off_u_mm) || !std::isfinite(geom->off_v_mm))
        return set_error(CYL_EINVAL, "detector offset must be finite");
    if (!geom->angles_rad) return set_error(CYL_EINVAL, "angles_rad is null");
    for (int p = 0; p < geom->n_proj; ++p)
        if (!std::isfinite(geom->angles_rad[p])) return set_error(CYL_EINVAL, "non-finite angle");
    const double pv[6] = {pose->alpha, pose->beta, pose->gamma, pose->tx, pose->ty, pose->tz};
    for (double v : pv)
        if (!std::isfinite(v)) return set_error(CYL_EINVAL, "non-finite pose");
    // the grid cylinder must lie in front of the source for every view
    const double reach = std::sqrt(grid->radius_mm * grid->radius_mm +
                                   0.25 * grid->height_mm * grid->height_mm) +
                         std::sqrt(pose->tx * pose->tx + pose->ty * pose->ty + pose->tz * pose->tz);
    if (reach >= geom->sod_mm) return set_error(CYL_EINVAL, "the grid cylinder reaches the source");
    return CYL_OK;
}

// Tiles: tt wedges (all of them when N_theta <= 16, else at most a quarter turn) x th
// slabs, sized so that the back-projection's two FP32 accumulators of a tile take about
// 96 KB of shared memory (two CTAs per SM).  CYL_TILE="tt,th" overrides the shape.
int choose_tiles(const cyl_grid &grid, int max_smem, TileDev &td)
{
    const int n_t = grid.n_theta, n_r = grid.n_r, n_h = grid.n_h;
    const int trig = (int)sizeof(float2) * ((n_t + 1) & ~1);
    int tt = n_t <= 16 ? n_t : std::min(16, n_t / 4);
    int budget = 96 * 1024;
    int th = 0;
    if (const char *env = getenv("CYL_TILE")) {
        int a = 0, b = 0;
        if (sscanf(env, "%d,%d", &a, &b) == 2 && a >= 1 && b >= 1) {
            if (n_t > 16 && a <= n_t / 4) tt = a;
            th = std::min(b, n_h);
        }
    }
    while (tt > 1 && trig + 8LL * tt * n_r > max_smem && n_t > 16) tt /= 2;
    if (trig + 8LL * tt * n_r > max_smem)
        return set_error(CYL_EINVAL, "grid too fine in r / theta for one tile in shared memory");
    if (th == 0) th = (int)std::max<int64_t>(1, (budget - trig) / (8LL * tt * n_r));
    th = std::min(th, n_h);
    while (th > 1 && trig + 8LL * tt * th * n_r > max_smem) --th;
    td.tt = tt;
    td.th = th;
    td.n_tt = (n_t + tt - 1) / tt;
    td.n_th = (n_h + th - 1) / th;
    td.n_tiles = td.n_tt * td.n_th;
    td.smem_fp = trig + 4 * tt * th * n_r;
    td.smem_bp = trig + 8 * tt * th * n_r;
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
}

void build_views(const cyl_grid &grid, const cyl_geom &geom, const cyl_pose &pose,
                 const TileDev &td, std::vector<ProjGeom> &geo, std::vector<int4> &bbox)
{
    double R[3][3];
    alignment_matrix(pose, R);
    const double T[3] = {pose.tx, pose.ty, pose.tz};
    const int W = geom.det_w, H = geom.det_h;
    geo.resize(geom.n_proj);
    bbox.resize((size_t)geom.n_proj * td.n_tiles);
    const double xd = geom.sdd_mm - geom.sod_mm;
    const double u0 = -0.5 * (W - 1) * geom.pitch_u_mm + geom.off_u_mm;
    const double v0 = -0.5 * (H - 1) * geom.pitch_v_mm + geom.off_v_mm;
    const double dth = 2.0 * M_PI / grid.n_theta, dh = grid.height_mm / grid.n_h;
    for (int p = 0; p < geom.n_proj; ++p) {
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

        // object point -> fractional detector pixel (iu, iv); false if not in front
        auto to_pixel = [&](const double o[3], double &fu, double &fv) -> bool {
            double st[3];
            for (int i = 0; i < 3; ++i) st[i] = R[0][i] * o[0] + R[1][i] * o[1] + R[2][i] * o[2] + T[i];
            const double lx = c * st[0] - s * st[1], ly = s * st[0] + c * st[1], lz = st[2];
            const double den = lx + geom.sod_mm;
            if (!(den > 1e-9 * geom.sod_mm)) return false;
            fu = (geom.sdd_mm * ly / den - geom.off_u_mm) / geom.pitch_u_mm + 0.5 * (W - 1);
            fv = (geom.sdd_mm * lz / den - geom.off_v_mm) / geom.pitch_v_mm + 0.5 * (H - 1);
            return true;
        };
        for (int tile = 0; tile < td.n_tiles; ++tile) {
            const int tt = tile % td.n_tt, ht = tile / td.n_tt;
            const int t0 = tt * td.tt, t1 = std::min(t0 + td.tt, grid.n_theta);
            const int s0 = ht * td.th, s1 = std::min(s0 + td.th, grid.n_h);
            const double h_lo = -0.5 * grid.height_mm + s0 * dh, h_hi = -0.5 * grid.height_mm + s1 * dh;
            // convex hull of the tile in the x'y' plane
            double px[4], py[4];
            int npt;
            if (td.n_tt == 1) {
                const double r = grid.radius_mm * (1.0 + 1e-9);
                const double sq[4][2] = {{-r, -r}, {r, -r}, {r, r}, {-r, r}};
                for (int k = 0; k < 4; ++k) { px[k] = sq[k][0]; py[k] = sq[k][1]; }
                npt = 4;
            } else {
                const double ta = t0 * dth, tb = t1 * dth;
                const double rc = grid.radius_mm / cos(0.5 * (tb - ta)) * (1.0 + 1e-9);
                px[0] = 0.0; py[0] = 0.0;
                px[1] = rc * cos(ta); py[1] = rc * sin(ta);
                px[2] = rc * cos(tb); py[2] = rc * sin(tb);
                npt = 3;
            }
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            bool whole = false;
            for (int k = 0; k < npt && !whole; ++k)
                for (int e = 0; e < 2; ++e) {
                    const double o[3] = {px[k], py[k], e ? h_hi : h_lo};
                    double fu, fv;
                    if (!to_pixel(o, fu, fv)) { whole = true; break; }
                    umin = std::min(umin, fu); umax = std::max(umax, fu);
                    vmin = std::min(vmin, fv); vmax = std::max(vmax, fv);
                }
            int4 b;
            if (whole) {
                b = make_int4(0, 0, W - 1, H - 1);
            } else {
                const double lo_u = std::max(std::floor(umin) - 1.0, 0.0);
                const double hi_u = std::min(std::ceil(umax) + 1.0, (double)(W - 1));
                const double lo_v = std::max(std::floor(vmin) - 1.0, 0.0);
                const double hi_v = std::min(std::ceil(vmax) + 1.0, (double)(H - 1));
                if (lo_u > hi_u || lo_v > hi_v) b = make_int4(1, 1, 0, 0);
                else b = make_int4((int)lo_u, (int)lo_v, (int)hi_u, (int)hi_v);
            }
            bbox[(size_t)p * td.n_tiles + tile] = b;
        }
    }
}

}  // namespace cylct
