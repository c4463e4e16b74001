// C ABI of libcylct.so: plans, log transform, projection, back-projection, SART solve.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

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

bool valid_dtype(int t) { return t == CYL_F32 || t == CYL_F16 || t == CYL_BF16; }

int check_range(const cyl_plan *plan, int32_t p0, int32_t np)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (p0 < 0 || np < 0 || (int64_t)p0 + np > plan->geom.n_proj)
        return set_error(CYL_EINVAL, "projection range outside the plan");
    return CYL_OK;
}

}  // namespace

#define CYL_CUDA(call)                                           \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);     \
    } while (0)

namespace cylct {

int set_error(int code, const char *msg)
{
    snprintf(g_detail, sizeof g_detail, "%s", msg);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    return fail(CYL_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace cylct

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

extern "C" int cyl_binary_version(int device, int32_t *binary_version)
{
    if (!binary_version) return set_error(CYL_EINVAL, "binary_version is null");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return set_error(CYL_EDEVICE, "no such CUDA device");
    }
    DeviceGuard dg(device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    int v = 0;
    const cudaError_t e = kernel_binary_version(&v);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_error(e, "cudaFuncGetAttributes");
    }
    *binary_version = v;
    return CYL_OK;
}

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
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    cyl_plan *pl = new (std::nothrow) cyl_plan();
    if (!pl) return set_error(CYL_ENOMEM, "host allocation failed");
    rc = pl->init(*grid, *geom, *pose, device);
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
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    cudaStream_t user = (cudaStream_t)stream;
    CYL_CUDA(cudaEventRecord(plan->ev_in, user));
    CYL_CUDA(cudaStreamWaitEvent(plan->ws, plan->ev_in, 0));
    if ((rc = plan->upload_pose(*pose, plan->ws))) return rc;
    CYL_CUDA(cudaEventRecord(plan->ev_out, plan->ws));
    CYL_CUDA(cudaStreamWaitEvent(user, plan->ev_out, 0));
    return CYL_OK;
}

extern "C" int cyl_plan_destroy(cyl_plan *plan)
{
    if (!plan) return CYL_OK;
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    delete plan;
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

extern "C" int cyl_row_sums(cyl_plan *plan, int32_t p0, int32_t np, float *L_out, void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (np == 0) return CYL_OK;
    if (!L_out) return set_error(CYL_EINVAL, "L_out is null");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    cudaError_t e = launch_row_sums(plan->scan_dev(), p0, np, L_out, (cudaStream_t)stream, plan->ray_list());
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
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    const size_t n = (size_t)np * plan->n_pix;
    float *q = static_cast<float *>(sino_out);
    if (sino_dtype != CYL_F32) {
        if ((rc = plan->ensure((void **)&plan->d_q, plan->q_cap, sizeof(float) * n))) return rc;
        q = plan->d_q;
    }
    OnPlanStream ps{plan, (cudaStream_t)stream};
    CYL_CUDA(ps.begin());
    // the projector writes the rays of positive chord only
    if (plan->use_list) CYL_CUDA(cudaMemsetAsync(q, 0, sizeof(float) * n, plan->ws));
    CYL_CUDA(launch_fp_rays(plan->scan_dev(), plan->p_fp, p0, np, vol, vol_dtype, q, nullptr, 0, plan->ws,
                            plan->ray_list()));
    if (sino_dtype != CYL_F32)
        CYL_CUDA(launch_convert(q, CYL_F32, sino_out, sino_dtype, (int64_t)n, plan->ws));
    CYL_CUDA(ps.end());
    return CYL_OK;
}

extern "C" int cyl_backproject(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, int32_t p0,
                               int32_t np, float *vol_out, float *colsum_out, void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (!valid_dtype(sino_dtype)) return set_error(CYL_EINVAL, "bad dtype");
    if (!vol_out || (np > 0 && !sino)) return set_error(CYL_EINVAL, "null array");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    OnPlanStream ps{plan, (cudaStream_t)stream};
    CYL_CUDA(ps.begin());
    CYL_CUDA(cudaMemsetAsync(vol_out, 0, sizeof(float) * plan->n_vox, plan->ws));
    if (colsum_out) CYL_CUDA(cudaMemsetAsync(colsum_out, 0, sizeof(float) * plan->n_vox, plan->ws));
    CYL_CUDA(launch_bp_rays(plan->scan_dev(), plan->p_bp, p0, np, sino, sino_dtype, nullptr, nullptr,
                            vol_out, colsum_out, plan->ws, plan->ray_list()));
    CYL_CUDA(ps.end());
    return CYL_OK;
}

extern "C" int cyl_count_segments(cyl_plan *plan, int32_t p0, int32_t np, int64_t *counts_out,
                                  void *stream)
{
    int rc = check_range(plan, p0, np);
    if (rc) return rc;
    if (np == 0) return CYL_OK;
    if (!counts_out) return set_error(CYL_EINVAL, "counts_out is null");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    OnPlanStream ps{plan, (cudaStream_t)stream};
    CYL_CUDA(ps.begin());
    CYL_CUDA(cudaMemsetAsync(counts_out, 0, sizeof(int64_t) * np, plan->ws));
    CYL_CUDA(launch_count_rays(plan->scan_dev(), p0, np, reinterpret_cast<unsigned long long *>(counts_out),
                               plan->ws, plan->ray_list()));
    CYL_CUDA(ps.end());
    return CYL_OK;
}

extern "C" int cyl_plan_set_fused(cyl_plan *plan, int32_t enable)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    std::lock_guard<std::mutex> lock(plan->mu);
    plan->fused = enable != 0;
    plan->drop_graphs();
    return CYL_OK;
}

extern "C" int cyl_plan_set_sart_pieces(cyl_plan *plan, int32_t pieces)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (pieces != 0 && !valid_pieces(pieces)) return set_error(CYL_EINVAL, "pieces must be 1, 2, 4, 8 or 16");
    std::lock_guard<std::mutex> lock(plan->mu);
    plan->p_sart = pieces;
    plan->drop_graphs();
    return CYL_OK;
}

extern "C" int cyl_plan_set_records(cyl_plan *plan, int32_t enable, int32_t runs, void *stream)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (enable < 0 || enable > 2) return set_error(CYL_EINVAL, "enable must be 0, 1 or 2");
    int lg = 0;
    while (lg < 5 && (1 << lg) < runs) ++lg;
    if (runs != 0 && (runs < 0 || (1 << lg) != runs)) return set_error(CYL_EINVAL, "runs must be 0, 1, 2, 4, 8, 16 or 32");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    cudaStream_t user = (cudaStream_t)stream;
    CYL_CUDA(cudaEventRecord(plan->ev_in, user));
    CYL_CUDA(cudaStreamWaitEvent(plan->ws, plan->ev_in, 0));
    plan->rec_mode = enable;
    plan->rec_lgP = runs ? lg : kRecLgP;
    int rc = CYL_OK;
    if (enable == 0) plan->free_records();
    else rc = plan->build_records(plan->ws);
    if (rc) return rc;
    CYL_CUDA(cudaEventRecord(plan->ev_out, plan->ws));
    CYL_CUDA(cudaStreamWaitEvent(user, plan->ev_out, 0));
    return CYL_OK;
}

extern "C" int cyl_plan_records(const cyl_plan *plan, int32_t *ready, int64_t *rec_bytes, int32_t *gather,
                                int64_t *gather_bytes)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (ready) *ready = plan->rec_ready ? 1 : 0;
    if (rec_bytes) *rec_bytes = plan->rec_ready ? plan->rec_rows * 32 * (int64_t)sizeof(uint32_t) : 0;
    if (gather) *gather = plan->vox_ready ? 1 : 0;
    if (gather_bytes)
        *gather_bytes = plan->vox_ready ? plan->vox_entries * (int64_t)sizeof(uint2) +
                                              (plan->n_vox + 1) * plan->geom.n_proj * (int64_t)sizeof(uint32_t)
                                        : 0;
    return CYL_OK;
}

extern "C" int cyl_plan_tune(cyl_plan *plan, void *stream)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    cudaStream_t user = (cudaStream_t)stream;
    CYL_CUDA(cudaEventRecord(plan->ev_in, user));
    CYL_CUDA(cudaStreamWaitEvent(plan->ws, plan->ev_in, 0));
    int rc = plan->tune(plan->ws);
    if (rc) return rc;
    CYL_CUDA(cudaEventRecord(plan->ev_out, plan->ws));
    CYL_CUDA(cudaStreamWaitEvent(user, plan->ev_out, 0));
    return CYL_OK;
}

extern "C" int cyl_plan_get_pieces(const cyl_plan *plan, int32_t *fp, int32_t *bp)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (fp) *fp = plan->p_fp > 0 ? plan->p_fp : default_pieces(0);
    if (bp) *bp = plan->p_bp > 0 ? plan->p_bp : default_pieces(1);
    return CYL_OK;
}

extern "C" int cyl_plan_set_pieces(cyl_plan *plan, int32_t fp, int32_t bp)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if ((fp != 0 && !valid_pieces(fp)) || (bp != 0 && !valid_pieces(bp)))
        return set_error(CYL_EINVAL, "pieces must be 0, 1, 2, 4, 8 or 16");
    std::lock_guard<std::mutex> lock(plan->mu);
    plan->p_fp = fp;
    plan->p_bp = bp;
    plan->drop_graphs();
    return CYL_OK;
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

extern "C" int cyl_sart_solve(cyl_plan *plan, const void *sino, cyl_dtype sino_dtype, const void *x0,
                              const void *w, const cyl_sart_params *params, void *x_out,
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
    if (!valid_weight_dtype(params->weight_dtype)) return set_error(CYL_EINVAL, "bad weight dtype");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    std::lock_guard<std::mutex> lock(plan->mu);
    return plan->solve(sino, sino_dtype, x0, w, *params, x_out, x_dtype, (cudaStream_t)stream);
}
