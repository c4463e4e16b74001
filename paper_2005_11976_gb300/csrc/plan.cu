// Plan set-up and the SART solve driver (Eq. 7 over ordered subsets, n_iter sweeps).
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

int cyl_plan::init(const cyl_grid &gr, const cyl_geom &ge, const cyl_pose &po, int dev)
{
    device = dev;
    grid = gr;
    geom = ge;
    pose = po;
    if (ge.angles_rad) angles.assign(ge.angles_rad, ge.angles_rad + ge.n_proj);
    else angles.assign(ge.n_proj, 0.0);
    geom.angles_rad = angles.data();
    if (ge.frames_mm) {
        frames.assign(ge.frames_mm, ge.frames_mm + 12 * (size_t)ge.n_proj);
        geom.frames_mm = frames.data();
    }
    n_vox = (int64_t)gr.n_h * gr.n_theta * gr.n_r;
    n_pix = (int64_t)ge.det_w * ge.det_h;
    int rc;
    std::vector<float2> trig;
    build_grid(grid, geom, g, trig);
    const size_t n_rays = (size_t)geom.n_proj * n_pix;
    if ((rc = alloc(&d_geo, sizeof(ProjGeom) * geom.n_proj))) return rc;
    if ((rc = alloc(&d_trig, sizeof(float2) * trig.size()))) return rc;
    {   // compact or dense, fixed for the plan's life: the first pose decides
        std::vector<ProjGeom> geo;
        build_views(geom, pose, geo);
        use_list = n_rays < ((size_t)1 << 32) && hit_fraction_bound(grid, geom, geo) < 0.75;
    }
    if (use_list) {
        const size_t cpv = ((size_t)n_pix + kActChunk - 1) / kActChunk;
        if ((rc = alloc(&d_act_off, sizeof(int64_t) * (geom.n_proj + 1)))) return rc;
        if ((rc = alloc(&d_act_chunk, sizeof(int64_t) * cpv * geom.n_proj))) return rc;
    } else {
        for (int k = 0; k < 3; ++k)
            if ((rc = alloc(&d_ray[k], sizeof(float4) * n_rays))) return rc;
        if ((rc = alloc(&d_split, sizeof(uint16_t) * kSplit * n_rays))) return rc;
    }
    if ((rc = alloc(&d_sched, sizeof(int) * kSched))) return rc;
    for (int k = 0; k < 2; ++k)
        if ((rc = alloc(&d_nd[k], sizeof(float2) * n_vox))) return rc;
    if ((rc = alloc(&d_wscale, 2 * sizeof(float)))) return rc;
    PL_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
    PL_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    PL_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    PL_CUDA(cudaEventCreateWithFlags(&ev_geo, cudaEventDisableTiming));
    PL_CUDA(cudaMallocHost(&h_geo, sizeof(ProjGeom) * geom.n_proj));
    PL_CUDA(cudaMemcpyAsync(d_trig, trig.data(), sizeof(float2) * trig.size(), cudaMemcpyHostToDevice, ws));
    PL_CUDA(cudaMemsetAsync(d_sched, 0, sizeof(int) * kSched, ws));
    if ((rc = upload_pose(pose, ws))) return rc;
    PL_CUDA(cudaStreamSynchronize(ws));
    return CYL_OK;
}

int cyl_plan::upload_pose(const cyl_pose &po, cudaStream_t st)
{
    std::vector<ProjGeom> geo;
    build_views(geom, po, geo);
    // the pinned staging copies may still feed the previous upload
    PL_CUDA(cudaEventSynchronize(ev_geo));
    std::memcpy(h_geo, geo.data(), sizeof(ProjGeom) * geo.size());
    PL_CUDA(cudaMemcpyAsync(d_geo, h_geo, sizeof(ProjGeom) * geo.size(), cudaMemcpyHostToDevice, st));
    PL_CUDA(cudaEventRecord(ev_geo, st));
    if (!use_list) {
        PL_CUDA(launch_rays(g, d_geo, geom.n_proj, d_ray[0], d_ray[1], d_ray[2], st));
        // the cut walk also counts each ray's pieces when the pose keeps records
        const int64_t n_rays = (int64_t)geom.n_proj * n_pix;
        int rc;
        if (rec_mode && (rc = ensure((void **)&d_rcnt, rcnt_cap, sizeof(uint32_t) * n_rays))) return rc;
        PL_CUDA(launch_split(scan_dev(), n_rays, d_split, st, rec_mode ? d_rcnt : nullptr));
        if ((rc = build_records(st, rec_mode != 0))) return rc;
    } else if (d_act && po.alpha == pose.alpha && po.beta == pose.beta && po.tx == pose.tx &&
               po.ty == pose.ty && po.tz == pose.tz) {
        // a spin about the part's axis: the grid cylinder, and so the list, stay as they are
        PL_CUDA(launch_list_refill(g, d_geo, d_act, n_listed, d_ray[0], d_ray[1], d_ray[2], st));
        PL_CUDA(launch_split(scan_dev(), n_listed, d_split, st));
    } else {
        // count this pose's rays of positive chord, size the compact buffers, then list
        // them with their records and cut them
        PL_CUDA(launch_list_count(g, d_geo, geom.n_proj, d_act_chunk, d_act_off, st));
        int64_t n = 0;
        PL_CUDA(cudaMemcpyAsync(&n, d_act_off + geom.n_proj, sizeof n, cudaMemcpyDeviceToHost, st));
        PL_CUDA(cudaStreamSynchronize(st));
        const size_t want = (size_t)std::max<int64_t>(n, 1);
        if (want * sizeof(uint32_t) > act_cap) {
            const size_t room = want + want / 8 + 64;   // re-posed parts vary a little
            int rc;
            for (int k = 0; k < 3; ++k)
                if ((rc = ensure((void **)&d_ray[k], ray_cap[k], sizeof(float4) * room))) return rc;
            if ((rc = ensure((void **)&d_split, split_cap, sizeof(uint16_t) * kSplit * room))) return rc;
            if ((rc = ensure((void **)&d_act, act_cap, sizeof(uint32_t) * room))) return rc;
        }
        n_listed = n;
        PL_CUDA(launch_list_fill(g, d_geo, geom.n_proj, d_act_chunk, n, d_act, d_ray[0], d_ray[1], d_ray[2], st));
        PL_CUDA(launch_split(scan_dev(), n, d_split, st));
    }
    pose = po;
    return CYL_OK;
}

void cyl_plan::drop_graphs()
{
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gexec_odd) cudaGraphExecDestroy(gexec_odd);
    if (gexec_timed) cudaGraphExecDestroy(gexec_timed);
    gexec = gexec_odd = gexec_timed = nullptr;
}

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
        drop_graphs();               // a captured graph may point at the old buffer
    }
    int rc = alloc(p, nbytes);
    if (!rc) cap = nbytes;
    return rc;
}

void cyl_plan::release(void **p, size_t &cap)
{
    if (!*p) return;
    cudaStreamSynchronize(ws);
    auto it = std::find(allocs.begin(), allocs.end(), *p);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(*p);
    bytes -= cap;
    *p = nullptr;
    cap = 0;
    drop_graphs();
}

void cyl_plan::free_gather()
{
    release((void **)&d_vent, vent_cap);
    release((void **)&d_voff, voff_cap);
    release((void **)&d_vcnt, vcnt_cap);
    release((void **)&d_vcur, vcur_cap);
    release((void **)&d_vtsum, vtsum_cap);
    release((void **)&d_vebase, vebase_cap);
    vox_ready = false;
    vox_entries = 0;
}

void cyl_plan::free_records()
{
    free_gather();
    release((void **)&d_rinv, rinv_cap);
    release((void **)&d_den64, den64_cap);
    release((void **)&d_den32, den32_cap);
    release((void **)&d_num, num_cap);
    rinv_sub = 0;
    release((void **)&d_rec, rec_cap);
    release((void **)&d_rcnt, rcnt_cap);
    release((void **)&d_ridx0, ridx0_cap);
    release((void **)&d_rrow, rrow_cap);
    release((void **)&d_rbad, rbad_cap);
    rec_ready = false;
    rec_rows = 0;
}

int cyl_plan::build_records(cudaStream_t st, bool counted)
{
    // captured sweeps launch the record kernels with the buffers' addresses: they stay
    // valid while the records do (a reallocation drops them in ensure)
    const bool was = rec_ready, was_vox = vox_ready;
    rec_ready = false;
    vox_ready = false;
    rinv_sub = 0;             // the column sums belong to the pose
    int rc = write_records(st, counted);
    if (!rc && rec_ready && rec_mode == 1) rc = build_gather(st);
    else if (rec_mode != 1) free_gather();
    if (rec_ready != was || vox_ready != was_vox) drop_graphs();
    return rc;
}

int cyl_plan::write_records(cudaStream_t st, bool counted)
{
    if (!rec_mode || use_list) return CYL_OK;
    const int64_t n_rays = (int64_t)geom.n_proj * n_pix;
    const int64_t n_tasks = (int64_t)geom.n_proj * ((n_pix + 31) / 32);   // 32 rays per task
    int rc;
    if ((rc = ensure((void **)&d_rcnt, rcnt_cap, sizeof(uint32_t) * n_rays))) return rc;
    if ((rc = ensure((void **)&d_ridx0, ridx0_cap, sizeof(int32_t) * (n_rays << rec_lgP)))) return rc;
    if ((rc = ensure((void **)&d_rrow, rrow_cap, sizeof(int64_t) * (n_tasks + 1)))) return rc;
    if ((rc = ensure((void **)&d_rbad, rbad_cap, sizeof(int)))) return rc;
    if (counted) PL_CUDA(launch_rec_rows(scan_dev(), geom.n_proj, d_rcnt, d_rrow, st));
    else PL_CUDA(launch_rec_count(scan_dev(), geom.n_proj, rec_lgP, d_rcnt, d_rrow, st));
    int64_t rows = 0;
    PL_CUDA(cudaMemcpyAsync(&rows, d_rrow + n_tasks, sizeof rows, cudaMemcpyDeviceToHost, st));
    PL_CUDA(cudaStreamSynchronize(st));
    if (rows < 0 || rows > n_tasks * (int64_t)g.max_steps) return set_error(CYL_EDEVICE, "record rows out of range");
    const size_t need = (size_t)std::max<int64_t>(rows, 1) * 32 * sizeof(uint32_t);
    if (need > rec_cap) {
        // the records leave room for everything else: at most 40 % of the device, and
        // 1 GiB of it free afterwards; otherwise the subsets walk the rays
        size_t fr = 0, tot = 0;
        PL_CUDA(cudaMemGetInfo(&fr, &tot));
        if (need > tot / 10 * 4 || need + ((size_t)1 << 30) > fr + rec_cap) {
            release((void **)&d_rec, rec_cap);
            return CYL_OK;
        }
        if (ensure((void **)&d_rec, rec_cap, need + need / 16)) return CYL_OK;
    }
    PL_CUDA(cudaMemsetAsync(d_rbad, 0, sizeof(int), st));
    PL_CUDA(launch_rec_fill(scan_dev(), geom.n_proj, rec_lgP, d_rcnt, d_rrow, d_rec, d_ridx0, d_rbad, st));
    int bad = 1;
    PL_CUDA(cudaMemcpyAsync(&bad, d_rbad, sizeof bad, cudaMemcpyDeviceToHost, st));
    PL_CUDA(cudaStreamSynchronize(st));
    rec_rows = rows;
    rec_ready = bad == 0;
    return CYL_OK;
}

int cyl_plan::build_gather(cudaStream_t st)
{
    const int64_t nt = (n_vox + 2047) / 2048;
    const size_t off_bytes = sizeof(uint32_t) * (size_t)(n_vox + 1) * geom.n_proj;
    size_t fr = 0, tot = 0;
    PL_CUDA(cudaMemGetInfo(&fr, &tot));
    // the transpose takes about twice the records: keep records and transpose within half
    // of the device with 1 GiB free; otherwise the subsets replay with reductions
    const size_t recb = (size_t)rec_rows * 128;
    if (off_bytes > voff_cap && (off_bytes + ((size_t)1 << 30) > fr + voff_cap || recb + off_bytes > tot / 2)) {
        free_gather();
        return CYL_OK;
    }
    int rc;
    if ((rc = ensure((void **)&d_voff, voff_cap, off_bytes))) return rc;
    if ((rc = ensure((void **)&d_vcnt, vcnt_cap, sizeof(uint32_t) * n_vox))) return rc;
    if ((rc = ensure((void **)&d_vcur, vcur_cap, sizeof(uint32_t) * n_vox))) return rc;
    if ((rc = ensure((void **)&d_vtsum, vtsum_cap, sizeof(uint32_t) * nt))) return rc;
    if ((rc = ensure((void **)&d_vebase, vebase_cap, sizeof(int64_t) * (geom.n_proj + 1)))) return rc;
    const RecDev rd = rec_dev();
    PL_CUDA(launch_vox_count(rd, geom.n_proj, n_vox, d_vcnt, d_voff, d_vtsum, d_vebase, st));
    std::vector<int64_t> eb(geom.n_proj + 1);
    PL_CUDA(cudaMemcpyAsync(eb.data(), d_vebase, sizeof(int64_t) * eb.size(), cudaMemcpyDeviceToHost, st));
    PL_CUDA(cudaStreamSynchronize(st));
    const int64_t total = eb[geom.n_proj];
    const size_t ent_bytes = sizeof(uint2) * (size_t)std::max<int64_t>(total, 1);
    if (ent_bytes > vent_cap) {
        PL_CUDA(cudaMemGetInfo(&fr, &tot));
        if (ent_bytes + ((size_t)1 << 30) > fr + vent_cap || recb + off_bytes + ent_bytes > tot / 2) {
            free_gather();
            return CYL_OK;
        }
        if (ensure((void **)&d_vent, vent_cap, ent_bytes + ent_bytes / 16)) {
            free_gather();
            return CYL_OK;
        }
    }
    PL_CUDA(launch_vox_fill(rd, geom.n_proj, n_vox, d_voff, eb.data(), d_vcur, d_vent, st));
    vox_entries = total;
    vox_ready = true;
    return CYL_OK;
}

int cyl_plan::prepare_records(int subset, cudaStream_t st, int &rc)
{
    rc = CYL_OK;
    if (!rec_ready) return 0;
    if (vox_ready) return 2;   // the gather form needs no column sums of its own
    const int n_sub = (geom.n_proj + subset - 1) / subset;
    const size_t nv4 = (size_t)((n_vox + 3) / 4) * 4;
    if (rinv_sub != subset) {
        const size_t want = sizeof(float) * nv4 * n_sub;   // each subset's r padded to a multiple of 4
        if (want > rinv_cap) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            if (want + ((size_t)1 << 30) > fr + rinv_cap) return 0;   // walk instead
        }
        if (ensure((void **)&d_rinv, rinv_cap, want)) return 0;
        if ((rc = ensure((void **)&d_den32, den32_cap, sizeof(float) * nv4))) return 0;
        if (cudaMemsetAsync(d_den32, 0, sizeof(float) * nv4, st) != cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "cudaMemsetAsync");
            return 0;
        }
        if (subset > 1) {
            if ((rc = ensure((void **)&d_den64, den64_cap, sizeof(double) * nv4))) return 0;
            if (cudaMemsetAsync(d_den64, 0, sizeof(double) * nv4, st) != cudaSuccess) {
                rc = cuda_error(cudaGetLastError(), "cudaMemsetAsync");
                return 0;
            }
        }
        const RecDev rd = rec_dev();
        for (int k = 0; k < n_sub; ++k) {
            const int p0 = k * subset, np = std::min(subset, geom.n_proj - p0);
            const cudaError_t e =
                launch_rec_inv_den(rd, p0, np, n_vox, d_den32, d_den64, d_rinv + (size_t)k * nv4, st);
            if (e != cudaSuccess) {
                rc = cuda_error(e, "launch_rec_inv_den");
                return 0;
            }
        }
        rinv_sub = subset;
    }
    if ((rc = ensure((void **)&d_num, num_cap, sizeof(float) * nv4))) return 0;
    if (cudaMemsetAsync(d_num, 0, sizeof(float) * nv4, st) != cudaSuccess) {
        rc = cuda_error(cudaGetLastError(), "cudaMemsetAsync");
        return 0;
    }
    return 1;
}

cudaEvent_t *cyl_plan::next_events(int n)
{
    const size_t need = ev_used + (size_t)n;
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
    drop_graphs();
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_geo) cudaEventDestroy(ev_geo);
    if (h_geo) cudaFreeHost(h_geo);
    if (ws) cudaStreamDestroy(ws);
    for (void *p : allocs) cudaFree(p);
}

// One sweep.  Subset k of the sweep uses accumulator b = (parity + k) & 1: forward-
// project (the kernel also clears accumulator b ^ 1, which the previous subset's update
// has consumed), back-project the residuals into accumulator b, then apply Eq. 7.  Timed
// runs record an event before the forward projection, between the kernels and after the
// update.
int cyl_plan::queue_sweep(const SolveState &s, cudaStream_t st, bool timed, int parity)
{
    const ScanDev sd = scan_dev();
    UpdateArgs upd;
    upd.x32 = s.x32;
    upd.x16 = s.x16;
    upd.x16_t = s.x16_t;
    upd.strict16 = s.strict16;
    upd.w = s.w;
    upd.w_t = s.w_t;
    upd.wscale = s.w ? d_wscale : nullptr;
    upd.lambda = (float)s.lambda;
    upd.clamp = s.clamp;
    upd.den_eps = g.eps;
    // timing events captured into a graph must be external records to be timed
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (timed) PL_CUDA(cudaStreamIsCapturing(st, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    int k = 0;
    for (int p0 = 0; p0 < geom.n_proj; p0 += s.subset, ++k) {
        const int np = std::min(s.subset, geom.n_proj - p0);
        const int b = (parity + k) & 1;
        const void *sino_p = static_cast<const char *>(s.sino) + (size_t)p0 * n_pix * dtype_size(s.sino_t);
        cudaEvent_t *ev = timed ? next_events(4) : nullptr;
        if (timed && !ev) return set_error(CYL_EDEVICE, "event creation failed");
        if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[0], st, rec_flags));
        if (s.rec == 2) {
            // the records' forward replay writes the residuals; one pass over the voxels
            // gathers their back-projection and column sums and updates x
            PL_CUDA(launch_rec_sart(rec_dev(), p0, np, s.x_proj, s.x_proj_t, sino_p, s.sino_t, nullptr, d_q,
                                    d_sched + 8, st));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[1], st, rec_flags));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[2], st, rec_flags));
            PL_CUDA(launch_vox_sart(vox_dev(), p0, np, d_q, upd, st));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[3], st, rec_flags));
            continue;
        }
        if (s.rec == 1) {
            // the same subset replaying the pose's stored records into the numerator; the
            // update divides by the pose's column sums
            PL_CUDA(launch_rec_sart(rec_dev(), p0, np, s.x_proj, s.x_proj_t, sino_p, s.sino_t, d_num, nullptr,
                                    d_sched + 8, st));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[1], st, rec_flags));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[2], st, rec_flags));
            PL_CUDA(launch_update_rec(n_vox, d_num, d_rinv + (size_t)k * (((size_t)n_vox + 3) / 4 * 4), upd, st));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[3], st, rec_flags));
            continue;
        } else if (fused) {
            // projection, residual and back-projection in one launch; no back-projector time
            PL_CUDA(launch_sart_rays(sd, p_sart, p0, np, s.x_proj, s.x_proj_t, sino_p, s.sino_t, d_nd[b], d_nd[b ^ 1],
                                     n_vox, st, ray_list()));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[1], st, rec_flags));
        } else {
            PL_CUDA(launch_fp_rays(sd, p_fp, p0, np, s.x_proj, s.x_proj_t, d_q, d_nd[b ^ 1], n_vox, st,
                                   ray_list()));
            if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[1], st, rec_flags));
            PL_CUDA(launch_bp_rays(sd, p_bp, p0, np, sino_p, s.sino_t, d_q, d_nd[b], nullptr, nullptr, st,
                                   ray_list()));
        }
        if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[2], st, rec_flags));
        PL_CUDA(launch_update_nd(n_vox, d_nd[b], upd, st));
        if (ev) PL_CUDA(cudaEventRecordWithFlags(ev[3], st, rec_flags));
    }
    return CYL_OK;
}

int cyl_plan::solve(const void *sino, cyl_dtype sino_t, const void *x0, const void *w,
                    const cyl_sart_params &prm, void *x_out, cyl_dtype x_t, cudaStream_t user)
{
    const PtrKind ks = kind_of(sino), kx0 = kind_of(x0), kw = kind_of(w), kxo = kind_of(x_out);
    const bool any_host = ks == kHost || kx0 == kHost || kw == kHost || kxo == kHost;
    const size_t xb = dtype_size(x_t), sb = dtype_size(sino_t);
    const size_t sino_bytes = (size_t)geom.n_proj * n_pix * sb;
    const int subset = std::min(prm.subset_size, geom.n_proj);
    const int n_sub = (geom.n_proj + subset - 1) / subset;
    int rc;
    if ((rc = ensure((void **)&d_q, q_cap, sizeof(float) * (size_t)n_pix * subset))) return rc;

    PL_CUDA(cudaEventRecord(ev_in, user));
    PL_CUDA(cudaStreamWaitEvent(ws, ev_in, 0));

    // stage host inputs
    const void *d_sino = sino, *d_x0 = x0;
    const void *d_w = w;
    const cyl_dtype w_t = (cyl_dtype)prm.weight_dtype;
    const size_t wb = dtype_size(w_t);
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
        if ((rc = ensure(&d_stage[2], stage_cap[2], wb * n_vox))) return rc;
        PL_CUDA(cudaMemcpyAsync(d_stage[2], w, wb * n_vox, cudaMemcpyHostToDevice, ws));
        d_w = d_stage[2];
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
    s.w_t = w_t;
    s.lambda = prm.lambda;
    s.clamp = prm.clamp_nonneg ? 1 : 0;
    s.subset = subset;
    if (d_x0 && d_x0 != d_xo) PL_CUDA(cudaMemcpyAsync(d_xo, d_x0, xb * n_vox, cudaMemcpyDeviceToDevice, ws));
    if (!d_x0) PL_CUDA(cudaMemsetAsync(d_xo, 0, xb * n_vox, ws));
    if (x_t == CYL_F32) {
        s.x32 = (float *)d_xo;
        s.x_proj = d_xo;
        s.x_proj_t = CYL_F32;
    } else if (prm.strict_16bit) {
        // the iterate itself is 16-bit: the projector reads it, every update rounds it
        s.x16 = d_xo;
        s.x16_t = x_t;
        s.x_proj = d_xo;
        s.x_proj_t = x_t;
        s.strict16 = 1;
    } else {
        // 16-bit storage of the warm start and the result around an FP32 iterate, which
        // the projector reads; the result is rounded once, after the last sweep
        if ((rc = ensure((void **)&d_x32, x32_cap, sizeof(float) * n_vox))) return rc;
        s.x32 = d_x32;
        s.x_proj = d_x32;
        s.x_proj_t = CYL_F32;
        PL_CUDA(launch_convert(d_xo, x_t, d_x32, CYL_F32, n_vox, ws));
    }
    if (d_w) PL_CUDA(launch_weight_scale(d_w, w_t, n_vox, prm.weight_mode, (float)prm.lambda, d_wscale, ws));
    s.rec = fused ? prepare_records(subset, ws, rc) : 0;
    if (rc) return rc;
    if (!s.rec)
        for (int k = 0; k < 2; ++k) PL_CUDA(cudaMemsetAsync(d_nd[k], 0, sizeof(float2) * n_vox, ws));

    const bool one_graph = !(n_sub & 1) || prm.n_iter == 1;
    if (timing && prm.use_graph && prm.n_iter > 0 && one_graph) {
        // one captured sweep with its timing events: every launch re-records them, so
        // after the solve they hold the kernel times of the last sweep
        if (!gexec_timed || !(gkey_timed == s)) {
            if (gexec_timed) cudaGraphExecDestroy(gexec_timed);
            gexec_timed = nullptr;
            ev_used = 0;
            cudaGraph_t graph = nullptr;
            PL_CUDA(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
            rc = queue_sweep(s, ws, true, 0);
            cudaError_t ce = cudaStreamEndCapture(ws, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&gexec_timed, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
            gkey_timed = s;
            ev_timed = ev_used;
        }
        ev_used = ev_timed;
        for (int it = 0; it < prm.n_iter; ++it) PL_CUDA(cudaGraphLaunch(gexec_timed, ws));
    } else if (timing) {
        ev_used = 0;
        for (int it = 0; it < prm.n_iter; ++it)
            if ((rc = queue_sweep(s, ws, true, (it * n_sub) & 1))) return rc;
    } else if (prm.use_graph && prm.n_iter > 0) {
        // one captured sweep per start parity; with an odd number of subsets the sweeps
        // alternate between the two
        const bool two = (n_sub & 1) && prm.n_iter > 1;
        if (!gexec || (two && !gexec_odd) || !(gkey == s)) {
            drop_graphs();
            for (int par = 0; par < (two ? 2 : 1); ++par) {
                cudaGraph_t graph = nullptr;
                PL_CUDA(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
                rc = queue_sweep(s, ws, false, par);
                cudaError_t ce = cudaStreamEndCapture(ws, &graph);
                if (rc) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
                cudaGraphExec_t ex = nullptr;
                ce = cudaGraphInstantiate(&ex, graph, 0);
                cudaGraphDestroy(graph);
                if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
                (par ? gexec_odd : gexec) = ex;
            }
            gkey = s;
        }
        for (int it = 0; it < prm.n_iter; ++it)
            PL_CUDA(cudaGraphLaunch(((it * n_sub) & 1) ? gexec_odd : gexec, ws));
    } else {
        for (int it = 0; it < prm.n_iter; ++it)
            if ((rc = queue_sweep(s, ws, false, (it * n_sub) & 1))) return rc;
    }

    if (x_t != CYL_F32 && !s.strict16) PL_CUDA(launch_convert(d_x32, CYL_F32, d_xo, x_t, n_vox, ws));
    if (kxo == kHost) PL_CUDA(cudaMemcpyAsync(x_out, d_xo, xb * n_vox, cudaMemcpyDeviceToHost, ws));
    PL_CUDA(cudaEventRecord(ev_out, ws));
    PL_CUDA(cudaStreamWaitEvent(user, ev_out, 0));
    if (any_host || timing) PL_CUDA(cudaStreamSynchronize(ws));
    if (timing) {
        for (int k = 0; k < 3; ++k) {
            kernel_ms[k] = 0.0;
            kernel_launches[k] = 0;
        }
        for (size_t base = 0; base + 4 <= ev_used; base += 4)
            for (int k = 0; k < 3; ++k) {
                if (fused && k == 1) continue;   // no separate back-projector launch
                float ms = 0.f;
                PL_CUDA(cudaEventElapsedTime(&ms, events[base + k], events[base + k + 1]));
                kernel_ms[k] += ms;
                kernel_launches[k] += 1;
            }
    }
    return CYL_OK;
}

// Autotuner: time the projector, the back-projector and the one-launch subset of view 0
// for 1, 2, 4, 8 and 16 pieces per ray and keep the fastest of each (the walk's cost does not depend on the
// volume's values, so a zero volume and zero data serve).
int cyl_plan::tune(cudaStream_t st)
{
    int rc;
    if ((rc = ensure((void **)&d_q, q_cap, sizeof(float) * (size_t)n_pix))) return rc;
    if ((rc = ensure((void **)&d_x32, x32_cap, sizeof(float) * n_vox))) return rc;
    PL_CUDA(cudaMemsetAsync(d_x32, 0, sizeof(float) * n_vox, st));
    PL_CUDA(cudaMemsetAsync(d_q, 0, sizeof(float) * n_pix, st));
    const ScanDev sd = scan_dev();
    cudaEvent_t e[2];
    PL_CUDA(cudaEventCreate(&e[0]));
    PL_CUDA(cudaEventCreate(&e[1]));
    float best_fp = 1e30f, best_bp = 1e30f, best_sart = 1e30f;
    for (int P = 1; P <= kSplit; P *= 2) {
        for (int kind = 0; kind < 3; ++kind) {
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                PL_CUDA(cudaEventRecord(e[0], st));
                if (kind == 0)
                    PL_CUDA(launch_fp_rays(sd, P, 0, 1, d_x32, CYL_F32, d_q, nullptr, 0, st, ray_list()));
                else if (kind == 1)
                    PL_CUDA(launch_bp_rays(sd, P, 0, 1, d_q, CYL_F32, d_q, d_nd[0], nullptr, nullptr, st, ray_list()));
                else
                    PL_CUDA(launch_sart_rays(sd, P, 0, 1, d_x32, CYL_F32, d_q, CYL_F32, d_nd[0], nullptr, 0, st,
                                             ray_list()));
                PL_CUDA(cudaEventRecord(e[1], st));
                PL_CUDA(cudaEventSynchronize(e[1]));
                float ms = 0.f;
                PL_CUDA(cudaEventElapsedTime(&ms, e[0], e[1]));
                ms_min = std::min(ms_min, ms);
            }
            if (kind == 0 && ms_min < best_fp) { best_fp = ms_min; p_fp = P; }
            if (kind == 1 && ms_min < best_bp) { best_bp = ms_min; p_bp = P; }
            if (kind == 2 && ms_min < best_sart) { best_sart = ms_min; p_sart = P; }
        }
    }
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
    PL_CUDA(cudaMemsetAsync(d_nd[0], 0, sizeof(float2) * n_vox, st));
    drop_graphs();
    return CYL_OK;
}
