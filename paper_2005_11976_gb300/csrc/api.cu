// C ABI of libcylct.so: plans, projection, back-projection, SART solve.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cylct_internal.h"
#include "plan.h"

using namespace cylct;

namespace {

thread_local char g_detail[256] = "";

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof g_detail, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(CYL_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

#define CYL_CUDA(call)                                           \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
    } while (0)

namespace cylct {

int set_error(int code, const char *msg)
{
    snprintf(g_detail, sizeof g_detail, "%s", msg);
    return code;
}

int cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

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
    if ((int64_t)grid->n_h * grid->n_theta * grid->n_r > (int64_t)1 << 31)
        return set_error(CYL_EINVAL, "grid larger than 2^31 voxels");
    if (!(grid->radius_mm > 0.0) || !(grid->height_mm > 0.0) || !std::isfinite(grid->radius_mm) ||
        !std::isfinite(grid->height_mm))
        return set_error(CYL_EINVAL, "grid radius and height must be finite and > 0");
    if (!(geom->sod_mm > 0.0) || !(geom->sdd_mm > geom->sod_mm) || !std::isfinite(geom->sdd_mm))
        return set_error(CYL_EINVAL, "need 0 < SOD < SDD");
    if (geom->n_proj < 1 || geom->det_w < 1 || geom->det_h < 1)
        return set_error(CYL_EINVAL, "projections and detector size must be >= 1");
    if ((int64_t)geom->det_w * geom->det_h > (int64_t)1 << 30)
        return set_error(CYL_EINVAL, "detector larger than 2^30 pixels");
    if (!(geom->pitch_u_mm > 0.0) || !(geom->pitch_v_mm > 0.0))
        return set_error(CYL_EINVAL, "pixel pitch must be > 0");
    if (!std::isfinite(geom->off_u_mm) || !std::isfinite(geom->off_v_mm))
        return set_error(CYL_EINVAL, "detector offset must be finite");
    if (!geom->angles_rad) return set_error(CYL_EINVAL, "angles_rad is null");
    for (int p = 0; p < geom->n_proj; ++p)
        if (!std::isfinite(geom->angles_rad[p])) return set_error(CYL_EINVAL, "non-finite angle");
    const double pv[6] = {pose->alpha, pose->beta, pose->gamma, pose->tx, pose->ty, pose->tz};
    for (double v : pv)
        if (!std::isfinite(v)) return set_error(CYL_EINVAL, "non-finite pose");
    return CYL_OK;
}

// Host FP64 tables of one scan: per-projection ray geometry and the wedge trig table.
void build_tables(const cyl_grid &grid, const cyl_geom &geom, const cyl_pose &pose,
                  std::vector<ProjGeom> &geo, std::vector<float2> &trig, GridDev &g)
{
    double R[3][3];
    alignment_matrix(pose, R);
    const double T[3] = {pose.tx, pose.ty, pose.tz};
    geo.resize(geom.n_proj);
    const double xd = geom.sdd_mm - geom.sod_mm;
    const double u0 = -0.5 * (geom.det_w - 1) * geom.pitch_u_mm + geom.off_u_mm;
    const double v0 = -0.5 * (geom.det_h - 1) * geom.pitch_v_mm + geom.off_v_mm;
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
    }
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
    g.inv_dth = (float)(grid.n_theta / (2.0 * M_PI));
    g.dh = (float)(grid.height_mm / grid.n_h);
    g.inv_dh = (float)(grid.n_h / grid.height_mm);
    g.h0 = (float)(-0.5 * grid.height_mm);
}

}  // namespace cylct

// ------------------------------------------------------------------------- helpers

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool valid_dtype(int t) { return t == CYL_F32 || t == CYL_F16 || t == CYL_BF16; }

}  // namespace

// ----------------------------------------------------------------------------- ABI

extern "C" const char *cyl_last_error_detail(void) { return g_detail; }

extern "C" const char *cyl_strerror(int code)
{
    switch (code) {
    case CYL_OK: return "CYL_OK";
    case CYL_EINVAL: return "CYL_EINVAL";
    case CYL_ENOMEM: return "CYL_ENOMEM";
    case CYL_EDEVICE: return "CYL_EDEVICE";
    case CYL_EADMIT: return "CYL_EADMIT";
    case CYL_ETIMEOUT: return "CYL_ETIMEOUT";
    case CYL_ENOTFOUND: return "CYL_ENOTFOUND";
    case CYL_EPENDING: return "CYL_EPENDING";
    case CYL_ECANCELLED: return "CYL_ECANCELLED";
    }
    return "CYL_E?";
}

extern "C" const char *cyl_version(void) { return "cylct 1.0"; }

extern "C" int cyl_plan_create(const cyl_grid *grid, const cyl_geom *geom, const cyl_pose *pose,
                               int device, cyl_plan **out)
{
    if (!out) return set_error(CYL_EINVAL, "out is null");
    *out = nullptr;
    int rc = validate_scan(grid, geom, pose);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return set_error(CYL_EDEVICE, "no such CUDA device");
    }
    DeviceGuard dg(device);
    cyl_plan *pl = new (std::nothrow) cyl_plan();
    if (!pl) return set_error(CYL_ENOMEM, "host allocation failed");
    pl->device = device;
    pl->grid = *grid;
    pl->geom = *geom;
    pl->pose = *pose;
    pl->angles.assign(geom->angles_rad, geom->angles_rad + geom->n_proj);
    pl->geom.angles_rad = pl->angles.data();
    std::vector<ProjGeom> geo;
    std::vector<float2> trig;
    build_tables(pl->grid, pl->geom, pl->pose, geo, trig, pl->g);
    pl->n_vox = (int64_t)grid->n_h * grid->n_theta * grid->n_r;
    pl->n_pix = (int64_t)geom->det_w * geom->det_h;
    rc = pl->alloc(&pl->d_geo, sizeof(ProjGeom) * geo.size());
    if (!rc) rc = pl->alloc(&pl->d_trig, sizeof(float2) * trig.size());
    if (!rc) rc = pl->alloc(&pl->d_wscale, 2 * sizeof(float));
    if (!rc) rc = pl->alloc(&pl->d_counts, sizeof(unsigned long long) * geom->n_proj);
    if (!rc) rc = pl->alloc(&pl->d_num, sizeof(float) * pl->n_vox);
    if (!rc) rc = pl->alloc(&pl->d_den, sizeof(float) * pl->n_vox);
    if (!rc && cudaStreamCreateWithFlags(&pl->ws, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(CYL_EDEVICE, "stream creation failed");
    if (!rc && (cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&pl->ev_geo, cudaEventDisableTiming) != cudaSuccess))
        rc = set_error(CYL_EDEVICE, "event creation failed");
    if (!rc && cudaMallocHost(&pl->h_geo, sizeof(ProjGeom) * geo.size()) != cudaSuccess)
        rc = set_error(CYL_ENOMEM, "pinned allocation failed");
    if (!rc && cudaMemcpy(pl->d_geo, geo.data(), sizeof(ProjGeom) * geo.size(),
                          cudaMemcpyHostToDevice) != cudaSuccess)
        rc = set_error(CYL_EDEVICE, "table upload failed");
    if (!rc && cudaMemcpy(pl->d_trig, trig.data(), sizeof(float2) * trig.size(),
                          cudaMemcpyHostToDevice) != cudaSuccess)
        rc = set_error(CYL_EDEVICE, "table upload failed");
    if (rc) {
        delete pl;
        return rc;
    }
    *out = pl;
    return CYL_OK;
}

extern "C" int cyl_plan_set_pose(cyl_plan *plan, const cyl_pose *pose, void *stream)
{
    if (!plan || !pose) return set_error(CYL_EINVAL, "plan or pose is null");
    int rc = validate_scan(&plan->grid, &plan->geom, pose);
    if (rc) return rc;
    DeviceGuard dg(plan->device);
    std::lock_guard<std::mutex> lock(plan->mu);
    std::vector<ProjGeom> geo;
    std::vector<float2> trig;
    GridDev g;
    build_tables(plan->grid, plan->geom, *pose, geo, trig, g);
    // the pinned staging copy may still feed the previous upload
    CYL_CUDA(cudaEventSynchronize(plan->ev_geo));
    std::memcpy(plan->h_geo, geo.data(), sizeof(ProjGeom) * geo.size());
    cudaStream_t user = (cudaStream_t)stream;
    CYL_CUDA(cudaEventRecord(plan->ev_in, user));
    CYL_CUDA(cudaStreamWaitEvent(plan->ws, plan->ev_in, 0));
    CYL_CUDA(cudaMemcpyAsync(plan->d_geo, plan->h_geo, sizeof(ProjGeom) * geo.size(),
                             cudaMemcpyHostToDevice, plan->ws));
    CYL_CUDA(cudaEventRecord(plan->ev_geo, plan->ws));
    CYL_CUDA(cudaStreamWaitEvent(user, plan->ev_geo, 0));
    plan->pose = *pose;
    return CYL_OK;
}

extern "C" int cyl_plan_destroy(cyl_plan *plan)
{
    if (!plan) return CYL_OK;
    {
        DeviceGuard dg(plan->device);
        delete plan;
    }
    return CYL_OK;
}

extern "C" int cyl_plan_sizes(const cyl_plan *plan, int64_t *n_vox, int64_t *n_pix, int32_t *n_proj,
                              int64_t *device_bytes)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (n_vox) *n_vox = plan->n_vox;
    if (n_pix) *n_pix = plan->n_pix;
    if (n_proj) *n_proj = plan->geom.n_proj;
    if (device_bytes) *device_bytes = (int64_t)plan->bytes;
    return CYL_OK;
}

extern "C" int cyl_log_transform(const void *counts, cyl_dtype in, double i0, void *p_out,
                                 cyl_dtype out, int64_t n, void *stream)
{
    if (!valid_dtype(in) || !valid_dtype(out)) return set_error(CYL_EINVAL, "bad dtype");
    if (n < 0) return set_error(CYL_EINVAL, "n < 0");
    if (n == 0) return CYL_OK;
    if (!counts || !p_out) return set_error(CYL_EINVAL, "null array");
    if (!(i0 > 0.0) || !std::isfinite(i0)) return set_error(CYL_EINVAL, "I0 must be > 0");
    if (counts == p_out && in != out) return set_error(CYL_EINVAL, "in-place needs equal dtypes");
    cudaError_t e = launch_log(counts, in, i0, p_out, out, n, (cudaStream_t)stream);
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "log transform");
}

static int check_range(const cyl_plan *plan, int32_t p0, int32_t np)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (p0 < 0 || np < 0 || (int64_t)p0 + np > plan->geom.n_proj)
        return set_error(CYL_EINVAL, "projection range outside the plan");
    return CYL_OK;
}

extern "C" int cyl_row_sums(cyl_plan *plan, int32_t p0, int32_t np, float *L_out, void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (np == 0) return CYL_OK;
    if (!L_out) return set_error(CYL_EINVAL, "L_out is null");
    DeviceGuard dg(plan->device);
    cudaError_t e = launch_row_sums(plan->g, plan->d_geo, p0, np, L_out, (cudaStream_t)stream);
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "row sums");
}

extern "C" int cyl_project(cyl_plan *plan, const void *vol, cyl_dtype vol_dtype, int32_t p0,
                           int32_t np, void *sino_out, cyl_dtype sino_dtype, void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (!valid_dtype(vol_dtype) || !valid_dtype(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (np == 0) return CYL_OK;
    if (!vol || !sino_out) return set_error(CYL_EINVAL, "null array");
    DeviceGuard dg(plan->device);
    cudaError_t e = launch_project(plan->g, plan->d_geo, plan->d_trig, p0, np, vol, vol_dtype,
                                   sino_out, sino_dtype, plan->tile, (cudaStream_t)stream);
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "project");
}

extern "C" int cyl_backproject(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, int32_t p0,
                               int32_t np, float *vol_out, float *colsum_out, void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (!valid_dtype(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!vol_out || (np > 0 && !sino)) return set_error(CYL_EINVAL, "null array");
    DeviceGuard dg(plan->device);
    cudaStream_t st = (cudaStream_t)stream;
    CYL_CUDA(cudaMemsetAsync(vol_out, 0, sizeof(float) * plan->n_vox, st));
    if (colsum_out) CYL_CUDA(cudaMemsetAsync(colsum_out, 0, sizeof(float) * plan->n_vox, st));
    cudaError_t e = launch_backproject(plan->g, plan->d_geo, plan->d_trig, p0, np, sino,
                                       sino_dtype, vol_out, colsum_out, plan->tile, st);
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "backproject");
}

extern "C" int cyl_count_segments(cyl_plan *plan, int32_t p0, int32_t np, int64_t *counts_out,
                                  void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (np == 0) return CYL_OK;
    if (!counts_out) return set_error(CYL_EINVAL, "counts_out is null");
    DeviceGuard dg(plan->device);
    cudaStream_t st = (cudaStream_t)stream;
    CYL_CUDA(cudaMemsetAsync(counts_out, 0, sizeof(int64_t) * np, st));
    cudaError_t e = launch_count(plan->g, plan->d_geo, plan->d_trig, p0, np,
                                 reinterpret_cast<unsigned long long *>(counts_out), plan->tile, st);
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "count segments");
}

extern "C" int cyl_plan_set_timing(cyl_plan *plan, int enable)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    plan->timing = enable != 0;
    return CYL_OK;
}

extern "C" int cyl_plan_kernel_time(cyl_plan *plan, int kind, double *ms_total, int64_t *launches)
{
    if (!plan || kind < 0 || kind > 2) return set_error(CYL_EINVAL, "bad plan or kind");
    if (ms_total) *ms_total = plan->kernel_ms[kind];
    if (launches) *launches = plan->kernel_launches[kind];
    return CYL_OK;
}

// --------------------------------------------------------------------- SART solve

namespace cylct {

// Queue one sweep (all subsets) of SART on stream st.  x_proj is the volume the
// projector reads (FP32 iterate, or its 16-bit copy / strict 16-bit iterate).
int queue_sweep(cyl_plan *pl, const SolveState &s, cudaStream_t st, bool timed)
{
    const int n_proj = pl->geom.n_proj;
    const int ss = s.subset;
    for (int p0 = 0; p0 < n_proj; p0 += ss) {
        const int np = n_proj - p0 < ss ? n_proj - p0 : ss;
        const void *sino_p = static_cast<const char *>(s.sino) +
                             (size_t)p0 * pl->n_pix * dtype_size(s.sino_t);
        cudaEvent_t *ev = timed ? pl->next_events(3) : nullptr;
        if (ev) CYL_CUDA(cudaEventRecord(ev[0], st));
        CYL_CUDA(launch_residual(pl->g, pl->d_geo, pl->d_trig, p0, np, s.x_proj, s.x_proj_t, sino_p,
                                 s.sino_t, pl->n_pix, pl->d_res, pl->tile, st));
        if (ev) CYL_CUDA(cudaEventRecord(ev[1], st));
        CYL_CUDA(launch_backproject(pl->g, pl->d_geo, pl->d_trig, p0, np, pl->d_res, CYL_F32,
                                    pl->d_num, pl->d_den, pl->tile, st));
        if (ev) CYL_CUDA(cudaEventRecord(ev[2], st));
        CYL_CUDA(launch_update(pl->n_vox, s.x32, s.x16, s.x16_t, s.strict16, pl->d_num, pl->d_den,
                               s.w, s.w ? pl->d_wscale : nullptr, (float)s.lambda, s.clamp, st));
        if (ev) CYL_CUDA(cudaEventRecord(ev[3], st));
    }
    return CYL_OK;
}

}  // namespace cylct

extern "C" int cyl_sart_solve(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, const void *x0,
                              const float *w, const cyl_sart_params *params, void *x_out,
                              cyl_dtype x_dtype, void *stream)
{
    if (!plan || !params) return set_error(CYL_EINVAL, "plan or params is null");
    if (!sino || !x_out) return set_error(CYL_EINVAL, "sino and x_out are required");
    if (!valid_dtype(sino_dtype) || !valid_dtype(x_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (params->n_iter < 0 || params->subset_size < 1)
        return set_error(CYL_EINVAL, "need n_iter >= 0 and subset_size >= 1");
    if (!std::isfinite(params->lambda)) return set_error(CYL_EINVAL, "lambda must be finite");
    if (params->weight_mode != 0 && params->weight_mode != 1)
        return set_error(CYL_EINVAL, "weight_mode must be 0 or 1");
    DeviceGuard dg(plan->device);
    cudaStream_t user = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(plan->mu);
    return plan->solve(sino, sino_dtype, x0, w, *params, x_out, x_dtype, user);
}
