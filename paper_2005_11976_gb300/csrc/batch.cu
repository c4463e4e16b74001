// Batched SART: many scans (own pose, own projection count) reconstructed together.
//
// Every scan runs exactly the subsets of its own cyl_sart_solve (Eq. 7, n_iter sweeps in
// index order); a round advances each unfinished scan by one subset.  A round is three
// kernels: the forward projection of the scans' current subsets and the back-projection
// into each scan's (numerator, column sum) accumulator, both persistent grids that take
// ray pieces of all the round's scans from one work counter, and the voxel update.  The
// rounds are queued once into a CUDA graph and launched as a single graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "plan.h"

using namespace cylct;

#define BT_CUDA(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);    \
    } while (0)

namespace {

bool on_device(const void *p, int dev)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

namespace cylct {

// Work list of a batched solve: per round, the (scan, subset) items.  Exposed for the
// serving scheduler, which builds its rounds the same way.
void batch_rounds(const std::vector<int> &n_proj, int subset, int n_iter,
                  std::vector<BatchItem> &items, std::vector<int> &n_items, int &rounds)
{
    const int n = (int)n_proj.size();
    std::vector<int> per(n);
    rounds = 0;
    for (int i = 0; i < n; ++i) {
        const int n_sub = (n_proj[i] + subset - 1) / subset;
        per[i] = n_iter * n_sub;
        rounds = std::max(rounds, per[i]);
    }
    items.assign((size_t)rounds * n, BatchItem{0, 0, 0, 0});
    n_items.assign(rounds, 0);
    for (int r = 0; r < rounds; ++r) {
        int k = 0;
        for (int i = 0; i < n; ++i) {
            if (r >= per[i]) continue;
            const int n_sub = (n_proj[i] + subset - 1) / subset;
            const int p0 = (r % n_sub) * subset;
            items[(size_t)r * n + k++] = BatchItem{i, p0, std::min(subset, n_proj[i] - p0), r & 1};
        }
        n_items[r] = k;
    }
}

}  // namespace cylct

namespace {

// Batched solve, or (tune) the batch autotuner: the same descriptors, then instead of the
// rounds, round 0's projector and back-projector timed for every piece setting; the
// fastest of each is stored in plans[0], whose settings the batch uses.  Tuning writes
// only the plans' scratch (projections and accumulators, cleared by every solve).
int batch_run(int32_t n, cyl_plan *const *plans, const void *const *sinos, cyl_dtype sino_dtype,
              const void *const *x0s, const void *const *ws, const cyl_sart_params *prm,
              void *const *x_outs, cyl_dtype x_dtype, void *stream, bool tune)
{
    if (n < 0 || (n > 0 && (!plans || !sinos || !x_outs)) || !prm)
        return set_error(CYL_EINVAL, "bad batch arguments");
    if (n > CYL_MAX_BATCH) return set_error(CYL_EINVAL, "more than CYL_MAX_BATCH scans");
    if (n == 0) return CYL_OK;
    if (sino_dtype < CYL_F32 || sino_dtype > CYL_BF16 || x_dtype < CYL_F32 || x_dtype > CYL_BF16)
        return set_error(CYL_EINVAL, "bad dtype");
    if (prm->n_iter < 0 || prm->subset_size < 1 || !std::isfinite(prm->lambda) ||
        (prm->weight_mode != 0 && prm->weight_mode != 1) || !valid_weight_dtype(prm->weight_dtype))
        return set_error(CYL_EINVAL, "bad SART parameters");
    const int dev = plans[0] ? plans[0]->device : -1;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || plans[i]->device != dev) return set_error(CYL_EINVAL, "plans must share one device");
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return set_error(CYL_EINVAL, "a plan appears twice in the batch");
        if (!sinos[i] || !x_outs[i]) return set_error(CYL_EINVAL, "sinogram and output are required");
    }
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (prev_dev != dev) cudaSetDevice(dev);
    struct Restore {
        int d;
        ~Restore() { if (d >= 0) cudaSetDevice(d); }
    } restore{prev_dev != dev ? prev_dev : -1};
    for (int i = 0; i < n; ++i)
        if (!on_device(sinos[i], dev) || !on_device(x_outs[i], dev) ||
            !on_device(x0s ? x0s[i] : nullptr, dev) || !on_device(ws ? ws[i] : nullptr, dev))
            return set_error(CYL_EINVAL, "batched solves take device arrays on the plans' device");
    {   // a round counts its warp tasks in 32 bits (bound: 16 pieces per ray)
        int64_t tasks = 0;
        for (int i = 0; i < n; ++i) {
            const int64_t sub = std::min<int64_t>(prm->subset_size, plans[i]->geom.n_proj);
            tasks += ((sub * plans[i]->n_pix + 31) / 32) * kSplit + kSplit;
        }
        if (tasks >= ((int64_t)1 << 31) - 1)
            return set_error(CYL_EINVAL, "batch too large: one round would exceed 2^31 warp tasks");
    }

    // lock the plans in address order
    std::vector<cyl_plan *> order(plans, plans + n);
    std::sort(order.begin(), order.end());
    std::vector<std::unique_lock<std::mutex>> locks;
    locks.reserve(n);
    for (cyl_plan *p : order) locks.emplace_back(p->mu);

    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t bs = plans[0]->ws;
    BT_CUDA(cudaEventRecord(plans[0]->ev_in, user));
    BT_CUDA(cudaStreamWaitEvent(bs, plans[0]->ev_in, 0));
    for (int i = 1; i < n; ++i) {   // earlier work of every plan (pose uploads, solves)
        BT_CUDA(cudaEventRecord(plans[i]->ev_out, plans[i]->ws));
        BT_CUDA(cudaStreamWaitEvent(bs, plans[i]->ev_out, 0));
    }

    const size_t xb = dtype_size(x_dtype);
    int rc;
    int64_t max_vox = 0;
    std::vector<BatchScan> scans(n);
    bool lists = false;   // some scan takes its tasks from its list of rays
    std::vector<int> n_proj(n);
    for (int i = 0; i < n; ++i) {
        cyl_plan *pl = plans[i];
        const int subset = std::min(prm->subset_size, pl->geom.n_proj);
        const size_t qlen = (size_t)subset * pl->n_pix;
        if ((rc = pl->ensure((void **)&pl->d_q, pl->q_cap, 2 * sizeof(float) * qlen))) return rc;
        for (int k = 0; k < 2; ++k) BT_CUDA(cudaMemsetAsync(pl->d_nd[k], 0, sizeof(float2) * pl->n_vox, bs));
        const void *x0 = x0s ? x0s[i] : nullptr;
        const void *w = ws ? ws[i] : nullptr;
        void *xo = x_outs[i];
        if (!tune && x0 && x0 != xo) BT_CUDA(cudaMemcpyAsync(xo, x0, xb * pl->n_vox, cudaMemcpyDeviceToDevice, bs));
        if (!tune && !x0) BT_CUDA(cudaMemsetAsync(xo, 0, xb * pl->n_vox, bs));
        BatchScan &sc = scans[i];
        sc.sd = pl->scan_dev();
        sc.rl = pl->ray_list();
        lists = lists || pl->use_list;
        sc.sino = sinos[i];
        sc.x_proj = xo;
        sc.q[0] = pl->d_q;
        sc.q[1] = pl->d_q + qlen;
        sc.q_len = (int64_t)qlen;
        sc.nd[0] = pl->d_nd[0];
        sc.nd[1] = pl->d_nd[1];
        sc.nd_len = pl->n_vox;
        max_vox = std::max(max_vox, pl->n_vox);
        UpdateArgs &u = sc.upd;
        u.x32 = nullptr;
        u.x16 = nullptr;
        u.x16_t = x_dtype;
        u.strict16 = 0;
        if (x_dtype == CYL_F32) {
            u.x32 = (float *)xo;
        } else if (prm->strict_16bit) {
            u.x16 = xo;
            u.strict16 = 1;
        } else {
            // FP32 iterate, read by the projector; rounded to x_dtype after the last round
            if ((rc = pl->ensure((void **)&pl->d_x32, pl->x32_cap, sizeof(float) * pl->n_vox))) return rc;
            u.x32 = pl->d_x32;
            sc.x_proj = pl->d_x32;
            if (!tune) BT_CUDA(launch_convert(xo, x_dtype, pl->d_x32, CYL_F32, pl->n_vox, bs));
        }
        u.w = w;
        u.w_t = (cyl_dtype)prm->weight_dtype;
        u.wscale = w ? pl->d_wscale : nullptr;
        u.lambda = (float)prm->lambda;
        u.clamp = prm->clamp_nonneg ? 1 : 0;
        u.den_eps = sc.sd.g.eps;
        if (w && !tune)
            BT_CUDA(launch_weight_scale(w, u.w_t, pl->n_vox, prm->weight_mode, (float)prm->lambda, pl->d_wscale,
                                        bs));
        n_proj[i] = pl->geom.n_proj;
    }
    std::vector<BatchItem> items;
    std::vector<int> n_items;
    int rounds = 0;
    batch_rounds(n_proj, prm->subset_size, tune ? 1 : prm->n_iter, items, n_items, rounds);

    if (rounds > 0) {
        void *d_blob = nullptr;
        const size_t b_scans = sizeof(BatchScan) * n, b_items = sizeof(BatchItem) * items.size(),
                     b_n = sizeof(int) * n_items.size();
        const size_t b_sched = sizeof(int) * kSched;
        BT_CUDA(cudaMallocAsync(&d_blob, b_sched + b_scans + b_items + b_n + 64, bs));
        char *base = static_cast<char *>(d_blob);
        int *d_sched = reinterpret_cast<int *>(base);
        BatchScan *d_scans = reinterpret_cast<BatchScan *>(base + ((b_sched + 15) & ~size_t(15)));
        BatchItem *d_items = reinterpret_cast<BatchItem *>(reinterpret_cast<char *>(d_scans) + ((b_scans + 15) & ~size_t(15)));
        int *d_n = reinterpret_cast<int *>(reinterpret_cast<char *>(d_items) + ((b_items + 15) & ~size_t(15)));
        BT_CUDA(cudaMemsetAsync(d_sched, 0, b_sched, bs));
        BT_CUDA(cudaMemcpyAsync(d_scans, scans.data(), b_scans, cudaMemcpyHostToDevice, bs));
        BT_CUDA(cudaMemcpyAsync(d_items, items.data(), b_items, cudaMemcpyHostToDevice, bs));
        BT_CUDA(cudaMemcpyAsync(d_n, n_items.data(), b_n, cudaMemcpyHostToDevice, bs));
        // projector and update types: the 16-bit iterate in strict mode, else FP32
        const bool strict = x_dtype != CYL_F32 && prm->strict_16bit;
        const cyl_dtype xt = strict ? x_dtype : CYL_F32, x16t = xt;
        // one launch per round for projection and back-projection when the first plan runs
        // its subsets so (cyl_plan_set_fused), with its pieces per ray
        const bool fused = plans[0]->fused;
        const int Pf = fused ? plans[0]->p_sart : plans[0]->p_fp, Pb = plans[0]->p_bp;
        const int round_parts = fused ? (kRoundFused | kRoundUpdate) : kRoundAll;
        if (tune) {
            cudaEvent_t e[2];
            BT_CUDA(cudaEventCreate(&e[0]));
            BT_CUDA(cudaEventCreate(&e[1]));
            float best[3] = {1e30f, 1e30f, 1e30f};
            int pick[3] = {0, 0, 0};
            const int tparts[3] = {kRoundFp, kRoundBp, kRoundFused};
            cudaError_t ce = cudaSuccess;
            for (int part = 0; part < 3 && ce == cudaSuccess; ++part)
                for (int P = 1; P <= kSplit && ce == cudaSuccess; P *= 2)
                    for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
                        ce = cudaEventRecord(e[0], bs);
                        if (ce == cudaSuccess)
                            ce = launch_batch_round(d_scans, d_items, d_n, n, 0, max_vox, P, P, tparts[part], d_sched,
                                                    xt, sino_dtype, x16t, bs, lists);
                        if (ce == cudaSuccess) ce = cudaEventRecord(e[1], bs);
                        if (ce == cudaSuccess) ce = cudaEventSynchronize(e[1]);
                        float ms = 0.f;
                        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e[0], e[1]);
                        if (ce == cudaSuccess && rep > 0 && ms < best[part]) {
                            best[part] = ms;
                            pick[part] = P;
                        }
                    }
            cudaEventDestroy(e[0]);
            cudaEventDestroy(e[1]);
            if (ce != cudaSuccess) return cuda_error(ce, "batch autotuner");
            plans[0]->p_fp = pick[0];
            plans[0]->p_bp = pick[1];
            plans[0]->p_sart = pick[2];
            plans[0]->drop_graphs();
        } else if (prm->use_graph) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            BT_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            for (int r = 0; r < rounds && ce == cudaSuccess; ++r)
                ce = launch_batch_round(d_scans, d_items, d_n, n, r, max_vox, Pf, Pb, round_parts, d_sched,
                                        xt, sino_dtype, x16t, bs, lists);
            cudaError_t ee = cudaStreamEndCapture(bs, &graph);
            if (ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_error(ce, "batched round launch");
            }
            if (ee != cudaSuccess) return cuda_error(ee, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
            ce = cudaGraphLaunch(exec, bs);
            cudaGraphExecDestroy(exec);      // released once the launch completes
            if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphLaunch");
        } else {
            for (int r = 0; r < rounds; ++r)
                BT_CUDA(launch_batch_round(d_scans, d_items, d_n, n, r, max_vox, Pf, Pb, round_parts, d_sched,
                                           xt, sino_dtype, x16t, bs, lists));
        }
        BT_CUDA(cudaFreeAsync(d_blob, bs));
    }
    if (!tune && x_dtype != CYL_F32 && !prm->strict_16bit)
        for (int i = 0; i < n; ++i)
            BT_CUDA(launch_convert(plans[i]->d_x32, CYL_F32, x_outs[i], x_dtype, plans[i]->n_vox, bs));
    BT_CUDA(cudaEventRecord(plans[0]->ev_out, bs));
    BT_CUDA(cudaStreamWaitEvent(user, plans[0]->ev_out, 0));
    for (int i = 1; i < n; ++i) BT_CUDA(cudaStreamWaitEvent(plans[i]->ws, plans[0]->ev_out, 0));
    for (int i = 0; i < n; ++i) {     // a captured single-scan graph may point at old buffers
        if (plans[i]->gexec) {
            cudaGraphExecDestroy(plans[i]->gexec);
            plans[i]->gexec = nullptr;
        }
    }
    return CYL_OK;
}

}  // namespace

extern "C" int cyl_sart_solve_batch(int32_t n, cyl_plan *const *plans, const void *const *sinos,
                                    cyl_dtype sino_dtype, const void *const *x0s,
                                    const void *const *ws, const cyl_sart_params *prm,
                                    void *const *x_outs, cyl_dtype x_dtype, void *stream)
{
    return batch_run(n, plans, sinos, sino_dtype, x0s, ws, prm, x_outs, x_dtype, stream, false);
}

extern "C" int cyl_sart_tune_batch(int32_t n, cyl_plan *const *plans, const void *const *sinos,
                                   cyl_dtype sino_dtype, const void *const *x0s,
                                   const void *const *ws, const cyl_sart_params *prm,
                                   void *const *x_outs, cyl_dtype x_dtype, void *stream)
{
    return batch_run(n, plans, sinos, sino_dtype, x0s, ws, prm, x_outs, x_dtype, stream, true);
}
