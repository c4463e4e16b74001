// SART solve driver of a plan (Eq. 6 over ordered subsets, n_iter sweeps).
#include <algorithm>
#include <cstring>

#include "plan.h"

using namespace cylct;

namespace {

enum PtrKind { kNull, kDevice, kHost };

PtrKind kind_of(const void *p)
{
    if (!p) return kNull;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kHost;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? kDevice : kHost;
}

}  // namespace

#define PL_CUDA(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);    \
    } while (0)

int cyl_plan::ensure(void **p, size_t &cap, size_t nbytes)
{
    if (*p && cap >= nbytes) return CYL_OK;
    if (*p) {
        cudaStreamSynchronize(ws);
        auto it = std::find(allocs.begin(), allocs.end(), *p);
        if (it != allocs.end()) allocs.erase(it);
        cudaFree(*p);
        bytes -= cap;
        *p = nullptr;
        cap = 0;
    }
    int rc = alloc(p, nbytes);
    if (!rc) cap = nbytes;
    return rc;
}

cudaEvent_t *cyl_plan::next_events(int n_kernels)
{
    const size_t need = ev_used + (size_t)n_kernels + 1;
    while (events.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        events.push_back(e);
    }
    cudaEvent_t *r = &events[ev_used];
    ev_used = need;
    return r;
}

cyl_plan::~cyl_plan()
{
    if (ws) cudaStreamSynchronize(ws);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_geo) cudaEventDestroy(ev_geo);
    if (h_geo) cudaFreeHost(h_geo);
    if (ws) cudaStreamDestroy(ws);
    for (void *p : allocs) cudaFree(p);
}

int cyl_plan::solve(const void *sino, cyl_dtype sino_t, const void *x0, const float *w,
                    const cyl_sart_params &prm, void *x_out, cyl_dtype x_t, cudaStream_t user)
{
    const PtrKind ks = kind_of(sino), kx0 = kind_of(x0), kw = kind_of(w), kxo = kind_of(x_out);
    const bool any_host = ks == kHost || kx0 == kHost || kw == kHost || kxo == kHost;
    const size_t xb = dtype_size(x_t), sb = dtype_size(sino_t);
    const size_t sino_bytes = (size_t)geom.n_proj * n_pix * sb;
    const int subset = std::min(prm.subset_size, geom.n_proj);
    int rc;
    if ((rc = ensure((void **)&d_res, res_cap, sizeof(float) * (size_t)n_pix * subset))) return rc;

    PL_CUDA(cudaEventRecord(ev_in, user));
    PL_CUDA(cudaStreamWaitEvent(ws, ev_in, 0));

    // stage host inputs
    const void *d_sino = sino, *d_x0 = x0;
    const float *d_w = w;
    if (ks == kHost) {
        if ((rc = ensure(&d_stage[0], stage_cap[0], sino_bytes))) return rc;
        PL_CUDA(cudaMemcpyAsync(d_stage[0], sino, sino_bytes, cudaMemcpyHostToDevice, ws));
        d_sino = d_stage[0];
    }
    if (kx0 == kHost) {
        if ((rc = ensure(&d_stage[1], stage_cap[1], xb * n_vox))) return rc;
        PL_CUDA(cudaMemcpyAsync(d_stage[1], x0, xb * n_vox, cudaMemcpyHostToDevice, ws));
        d_x0 = d_stage[1];
    }
    if (kw == kHost) {
        if ((rc = ensure(&d_stage[2], stage_cap[2], sizeof(float) * n_vox))) return rc;
        PL_CUDA(cudaMemcpyAsync(d_stage[2], w, sizeof(float) * n_vox, cudaMemcpyHostToDevice, ws));
        d_w = (const float *)d_stage[2];
    }
    void *d_xo = x_out;
    if (kxo == kHost) {
        if ((rc = ensure(&d_stage[3], stage_cap[3], xb * n_vox))) return rc;
        d_xo = d_stage[3];
    }

    // iterate buffers
    SolveState s;
    s.sino = d_sino;
    s.sino_t = sino_t;
    s.w = d_w;
    s.lambda = prm.lambda;
    s.clamp = prm.clamp_nonneg ? 1 : 0;
    s.subset = subset;
    if (x_t == CYL_F32) {
        s.x32 = (float *)d_xo;
        s.x_proj = d_xo;
        s.x_proj_t = CYL_F32;
        if (d_x0 && d_x0 != d_xo) PL_CUDA(cudaMemcpyAsync(d_xo, d_x0, xb * n_vox, cudaMemcpyDeviceToDevice, ws));
        if (!d_x0) PL_CUDA(cudaMemsetAsync(d_xo, 0, xb * n_vox, ws));
    } else {
        s.x16 = d_xo;
        s.x16_t = x_t;
        s.x_proj = d_xo;
        s.x_proj_t = x_t;
        s.strict16 = prm.strict_16bit ? 1 : 0;
        if (d_x0 && d_x0 != d_xo) PL_CUDA(cudaMemcpyAsync(d_xo, d_x0, xb * n_vox, cudaMemcpyDeviceToDevice, ws));
        if (!d_x0) PL_CUDA(cudaMemsetAsync(d_xo, 0, xb * n_vox, ws));
        if (!s.strict16) {
            if ((rc = ensure((void **)&d_x32, x32_cap, sizeof(float) * n_vox))) return rc;
            s.x32 = d_x32;
            PL_CUDA(launch_convert(d_xo, x_t, d_x32, CYL_F32, n_vox, ws));
        }
    }
    if (d_w) PL_CUDA(launch_weight_scale(d_w, n_vox, prm.weight_mode, (float)prm.lambda, d_wscale, ws));
    PL_CUDA(cudaMemsetAsync(d_num, 0, sizeof(float) * n_vox, ws));
    PL_CUDA(cudaMemsetAsync(d_den, 0, sizeof(float) * n_vox, ws));

    if (timing) {
        ev_used = 0;
        for (int it = 0; it < prm.n_iter; ++it)
            if ((rc = queue_sweep(this, s, ws, true))) return rc;
    } else if (prm.use_graph && prm.n_iter > 0) {
        if (!gexec || !(gkey == s)) {
            if (gexec) {
                cudaGraphExecDestroy(gexec);
                gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            PL_CUDA(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
            rc = queue_sweep(this, s, ws, false);
            cudaError_t ce = cudaStreamEndCapture(ws, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                gexec = nullptr;
                return cuda_error(ce, "cudaGraphInstantiate");
            }
            gkey = s;
        }
        for (int it = 0; it < prm.n_iter; ++it) PL_CUDA(cudaGraphLaunch(gexec, ws));
    } else {
        for (int it = 0; it < prm.n_iter; ++it)
            if ((rc = queue_sweep(this, s, ws, false))) return rc;
    }

    if (kxo == kHost) PL_CUDA(cudaMemcpyAsync(x_out, d_xo, xb * n_vox, cudaMemcpyDeviceToHost, ws));
    PL_CUDA(cudaEventRecord(ev_out, ws));
    PL_CUDA(cudaStreamWaitEvent(user, ev_out, 0));
    if (any_host || timing) PL_CUDA(cudaStreamSynchronize(ws));
    if (timing) {
        for (int k = 0; k < 3; ++k) {
            kernel_ms[k] = 0.0;
            kernel_launches[k] = 0;
        }
        const size_t per = 4;
        for (size_t base = 0; base + per <= ev_used; base += per)
            for (int k = 0; k < 3; ++k) {
                float ms = 0.f;
                PL_CUDA(cudaEventElapsedTime(&ms, events[base + k], events[base + k + 1]));
                kernel_ms[k] += ms;
                kernel_launches[k] += 1;
            }
    }
    return CYL_OK;
}
