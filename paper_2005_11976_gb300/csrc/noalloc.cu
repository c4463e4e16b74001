// Forward projection that allocates nothing: the FP32 accumulator lives in a fixed-size
// array in the library's static device memory instead of in plan scratch.
//
// For callers that must not allocate device memory while they run: a host framework that
// owns all of the device's memory through its own caching allocator, or an in-line
// inspection loop that cannot afford an allocation (and the synchronisation it can
// bring) between two parts.  cyl_project needs plan scratch for 16-bit outputs and
// allocates it on first use; cyl_project_noalloc never does.
#include <cmath>
#include <mutex>

#include "plan.h"

using namespace cylct;

namespace {

constexpr int64_t kNoAllocMaxElems = CYL_NOALLOC_MAX_ELEMS;   // 4 Mi floats = 16 MiB
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) float g_noalloc_acc[kNoAllocMaxElems];

std::mutex g_mu;
void *g_acc_ptr[kMaxDevices] = {};

// Device address of the array on `dev` (the current device), looked up once per device.
int acc_address(int dev, float **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_acc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
        if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress");
        g_acc_ptr[dev] = p;
    }
    *out = static_cast<float *>(g_acc_ptr[dev]);
    return CYL_OK;
}

}  // namespace

extern "C" int cyl_project_noalloc(cyl_plan *plan, const void *vol, cyl_dtype vol_dtype,
                                   int32_t p0, int32_t np, void *sino_out,
                                   cyl_dtype sino_dtype, void *stream)
{
    if (!plan) return set_error(CYL_EINVAL, "plan is null");
    if (p0 < 0 || np < 0 || (int64_t)p0 + np > plan->geom.n_proj)
        return set_error(CYL_EINVAL, "projection range outside the plan");
    if (vol_dtype < CYL_F32 || vol_dtype > CYL_BF16 || sino_dtype < CYL_F32 || sino_dtype > CYL_BF16)
        return set_error(CYL_EINVAL, "bad dtype");
    if (np == 0) return CYL_OK;
    if (!vol || !sino_out) return set_error(CYL_EINVAL, "null array");
    const int64_t n = (int64_t)np * plan->n_pix;
    if (n > kNoAllocMaxElems)
        return set_error(CYL_EINVAL, "np * H * W exceeds the allocation-free buffer (4 Mi values)");
    if (plan->device < 0 || plan->device >= kMaxDevices) return set_error(CYL_EINVAL, "device index");
    DeviceGuard dg(plan->device);
    if (!dg.ok) return cuda_error(dg.err, "cudaSetDevice");
    float *acc = nullptr;
    int rc = acc_address(plan->device, &acc);
    if (rc) return rc;
    // the plan's kernels run on its work stream, ordered after the caller's stream
    std::lock_guard<std::mutex> lock(plan->mu);
    OnPlanStream ps{plan, (cudaStream_t)stream};
    const cudaStream_t st = plan->ws;
    cudaError_t e = ps.begin();
    // the projector writes the rays of positive chord only: clear what the last call left
    if (e == cudaSuccess && plan->use_list) e = cudaMemsetAsync(acc, 0, sizeof(float) * n, st);
    if (e == cudaSuccess) e = launch_fp_rays(plan->scan_dev(), plan->p_fp, p0, np, vol, vol_dtype, acc, nullptr, 0, st,
                                              plan->ray_list());
    if (e == cudaSuccess) e = launch_convert(acc, CYL_F32, sino_out, sino_dtype, n, st);
    if (e == cudaSuccess) e = ps.end();
    return e == cudaSuccess ? CYL_OK : cuda_error(e, "cyl_project_noalloc");
}
