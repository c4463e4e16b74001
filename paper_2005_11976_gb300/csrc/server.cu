// Serving: continuous batching of inspection scans over the batched SART kernels.
//
// Requests queue on the host; a scheduler thread admits them when their device footprint
// fits the HBM budget (resident part data included), gives each a plan (re-posed from a
// pool of plans of the same part type and projection count when one is idle), and then
// runs rounds: every active scan advances by one SART subset per round (the same
// k_fp_batch / k_bp_batch kernels as cyl_sart_solve_batch).  Scans that arrive while
// others are on the GPU join at the next round; finished scans leave after their last
// round, their result is copied out, and their memory returns to the budget.
//
// Host waits are bounded: the scheduler polls CUDA events with a limit, so a stalled
// device turns into CYL_ETIMEOUT on the affected scans instead of a hung thread.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "plan.h"

using namespace cylct;

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr int64_t kWaitLimitNs = 120LL * 1000 * 1000 * 1000;   // one round, at most

struct Part {
    cyl_grid grid{};
    cyl_geom geom{};
    void *d_x0 = nullptr;       // warm start, storage dtype
    void *d_w = nullptr;        // weights (cfg.weight_dtype) or null
    float *d_wscale = nullptr;  // lambda / max(w) (or lambda)
    size_t bytes = 0;
    int64_t n_vox = 0;
};

struct Scan {
    uint64_t ticket = 0;
    cyl_request req{};
    std::vector<double> angles;
    int state = 0;              // 0 queued, 1 active, 2 finishing, 3 done
    int status = CYL_EPENDING;
    cyl_plan *plan = nullptr;
    void *d_sino = nullptr;     // device sinogram (own copy when the request's is host)
    bool own_sino = false;
    void *d_x = nullptr;        // device iterate / output (own when the request's is host)
    bool own_x = false;
    float *d_x32 = nullptr;     // FP32 iterate of 16-bit storage
    int n_sub = 0, rounds_total = 0, rounds_done = 0;
    size_t bytes = 0;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    cudaEvent_t done_ev = nullptr;
};

struct PlanKey {
    int part, n_proj;
    uint64_t angle_hash;
    bool operator<(const PlanKey &o) const
    {
        if (part != o.part) return part < o.part;
        if (n_proj != o.n_proj) return n_proj < o.n_proj;
        return angle_hash < o.angle_hash;
    }
};

uint64_t hash_angles(const std::vector<double> &a)
{
    uint64_t h = 1469598103934665603ULL;
    for (double v : a) {
        uint64_t b;
        std::memcpy(&b, &v, 8);
        h = (h ^ b) * 1099511628211ULL;
    }
    return h;
}

}  // namespace

struct cyl_server {
    cyl_server_cfg cfg{};
    cudaStream_t st = nullptr;
    std::mutex mu;
    std::condition_variable cv;        // wakes the scheduler
    std::condition_variable done_cv;   // wakes cyl_wait callers
    std::deque<Part> parts;            // deque: references stay valid as parts are added
    int64_t idle_bytes = 0;            // device bytes of pooled idle plans (in hbm_in_use)
    std::deque<std::shared_ptr<Scan>> queue;
    std::vector<std::shared_ptr<Scan>> active;
    std::map<uint64_t, std::shared_ptr<Scan>> tickets;
    std::multimap<PlanKey, cyl_plan *> idle_plans;
    uint64_t next_ticket = 1;
    int64_t hbm_in_use = 0;
    cyl_server_stats stats{};
    bool stop = false;
    std::thread thr;
    // round descriptors: pinned staging and device copies, one slot per round in flight
    int n_slots = 0;
    std::vector<void *> h_slot, d_slot;
    std::vector<cudaEvent_t> slot_ev;
    size_t slot_bytes = 0;
    int next_slot = 0;
    int *d_sched = nullptr;            // work counters of the round kernels (kSched)

    void footprint(const Part &pt, int n_proj, const double *angles, const cyl_pose &pose, size_t &plan_b,
                   size_t &scan_b) const;
    int admit(const std::shared_ptr<Scan> &s);
    void release(const std::shared_ptr<Scan> &s);
    void finish(const std::shared_ptr<Scan> &s, int status);
    bool wait_event(cudaEvent_t e);
    int run_round();
    void loop();
};

// Device bytes of one scan: its plan, dense (records and cuts of every ray) or compact (of
// the rays that can meet the grid, bounded from the pose exactly as the plan decides), and
// the scan's own buffers.
void cyl_server::footprint(const Part &pt, int n_proj, const double *angles, const cyl_pose &pose,
                           size_t &plan_b, size_t &scan_b) const
{
    const size_t npix = (size_t)pt.geom.det_w * pt.geom.det_h, n_rays = (size_t)n_proj * npix;
    const size_t sb = dtype_size(cfg.storage);
    const int subset = std::min(cfg.subset_size, n_proj);
    cyl_geom g = pt.geom;
    g.n_proj = n_proj;
    g.angles_rad = angles;
    std::vector<ProjGeom> geo;
    build_views(g, pose, geo);
    const double bound = hit_fraction_bound(pt.grid, g, geo);
    const size_t per_ray = 3 * sizeof(float4) + kSplit * sizeof(uint16_t);   // records, cuts
    size_t rays_b;
    if (n_rays < ((size_t)1 << 32) && bound < 0.75) {
        const size_t listed = (size_t)std::ceil(bound * (double)n_rays);
        const size_t room = listed + listed / 8 + 64;
        rays_b = room * (per_ray + sizeof(uint32_t)) +
                 ((size_t)n_proj * ((npix + kActChunk - 1) / kActChunk) + n_proj + 1) * sizeof(int64_t);
    } else {
        rays_b = n_rays * per_ray;
    }
    plan_b = rays_b + 2 * (size_t)subset * npix * sizeof(float)   // projection buffers
             + 2 * (size_t)pt.n_vox * sizeof(float2)               // (num, den) accumulators
             + (size_t)n_proj * sizeof(ProjGeom) + 64 * 1024;       // small tables
    scan_b = n_rays * sb                                             // sinogram
             + (size_t)pt.n_vox * sb                                 // iterate / output
             + (cfg.storage != CYL_F32 ? (size_t)pt.n_vox * sizeof(float) : 0);
}

bool cyl_server::wait_event(cudaEvent_t e)
{
    const int64_t t0 = now_ns();
    for (;;) {
        cudaError_t r = cudaEventQuery(e);
        if (r == cudaSuccess) return true;
        if (r != cudaErrorNotReady) return false;
        if (now_ns() - t0 > kWaitLimitNs) return false;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Give an admitted scan its plan and buffers; queue its input copies (server stream).
int cyl_server::admit(const std::shared_ptr<Scan> &s)
{
    Part &pt = parts[s->req.part];
    const int n_proj = s->req.n_proj;
    const PlanKey key{s->req.part, n_proj, hash_angles(s->angles)};
    auto it = idle_plans.find(key);
    int rc;
    if (it != idle_plans.end()) {
        s->plan = it->second;
        idle_plans.erase(it);
        if ((rc = cyl_plan_set_pose(s->plan, &s->req.pose, st))) return rc;
    } else {
        cyl_geom ge = pt.geom;
        ge.n_proj = n_proj;
        ge.angles_rad = s->angles.data();
        if ((rc = cyl_plan_create(&pt.grid, &ge, &s->req.pose, cfg.device, &s->plan))) return rc;
    }
    cyl_plan *pl = s->plan;
    const size_t sb = dtype_size(cfg.storage);
    const size_t sino_bytes = (size_t)n_proj * pl->n_pix * sb;
    const int subset = std::min(cfg.subset_size, n_proj);
    if ((rc = pl->ensure((void **)&pl->d_q, pl->q_cap, 2 * sizeof(float) * subset * pl->n_pix))) return rc;
    if (is_device(s->req.sino)) {
        s->d_sino = const_cast<void *>(s->req.sino);
    } else {
        if (cudaMallocAsync(&s->d_sino, sino_bytes, st) != cudaSuccess) return set_error(CYL_ENOMEM, "sinogram");
        s->own_sino = true;
        if (cudaMemcpyAsync(s->d_sino, s->req.sino, sino_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "sinogram upload");
    }
    if (is_device(s->req.x_out)) {
        s->d_x = s->req.x_out;
    } else {
        if (cudaMallocAsync(&s->d_x, (size_t)pl->n_vox * sb, st) != cudaSuccess) return set_error(CYL_ENOMEM, "volume");
        s->own_x = true;
    }
    if (pt.d_x0) {
        if (cudaMemcpyAsync(s->d_x, pt.d_x0, (size_t)pl->n_vox * sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "warm start copy");
    } else if (cudaMemsetAsync(s->d_x, 0, (size_t)pl->n_vox * sb, st) != cudaSuccess) {
        return set_error(CYL_EDEVICE, "volume clear");
    }
    if (cfg.storage != CYL_F32) {
        if (cudaMallocAsync(&s->d_x32, (size_t)pl->n_vox * sizeof(float), st) != cudaSuccess)
            return set_error(CYL_ENOMEM, "FP32 iterate");
        if (launch_convert(s->d_x, cfg.storage, s->d_x32, CYL_F32, pl->n_vox, st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "iterate conversion");
    }
    for (int k = 0; k < 2; ++k)
        if (cudaMemsetAsync(pl->d_nd[k], 0, sizeof(float2) * pl->n_vox, st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "back-projection accumulators");
    if (cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming) != cudaSuccess)
        return set_error(CYL_EDEVICE, "event");
    s->n_sub = (n_proj + subset - 1) / subset;
    s->rounds_total = cfg.n_iter * s->n_sub;
    s->rounds_done = 0;
    if (s->rounds_total == 0) {        // no sweep: the result is the warm start
        if (s->own_x && cudaMemcpyAsync(s->req.x_out, s->d_x, (size_t)pl->n_vox * sb,
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "result copy");
        if (cudaEventRecord(s->done_ev, st) != cudaSuccess) return set_error(CYL_EDEVICE, "event");
        s->state = 2;
    }
    return CYL_OK;
}

void cyl_server::release(const std::shared_ptr<Scan> &s)
{
    if (s->own_sino && s->d_sino) cudaFreeAsync(s->d_sino, st);
    if (s->own_x && s->d_x) cudaFreeAsync(s->d_x, st);
    if (s->d_x32) cudaFreeAsync(s->d_x32, st);
    s->d_sino = s->d_x = nullptr;
    s->d_x32 = nullptr;
    if (s->done_ev) {
        cudaEventDestroy(s->done_ev);
        s->done_ev = nullptr;
    }
    hbm_in_use -= (int64_t)s->bytes;
    if (s->plan) {
        if (s->status == CYL_OK) {
            int64_t pb = 0;
            cyl_plan_sizes(s->plan, nullptr, nullptr, nullptr, &pb);
            idle_plans.emplace(PlanKey{s->req.part, s->req.n_proj, hash_angles(s->angles)}, s->plan);
            idle_bytes += pb;
            hbm_in_use += pb;
        } else {
            cyl_plan_destroy(s->plan);
        }
        s->plan = nullptr;
    }
}

void cyl_server::finish(const std::shared_ptr<Scan> &s, int status)
{
    s->status = status;
    s->state = 3;
    s->t_done = now_ns();
    if (status == CYL_OK) ++stats.completed;
    else ++stats.failed;
    release(s);
    done_cv.notify_all();
}

// Queue one round for all active scans that still have subsets to run.
int cyl_server::run_round()
{
    std::vector<BatchScan> scans;
    std::vector<BatchItem> items;
    std::vector<std::shared_ptr<Scan>> members;
    int Pf = 0, Pb = 0, have_p = 0;
    bool fused = true;    // the round in one launch (as the first member's plan runs its subsets)
    bool lists = false;   // some member takes its tasks from its list of rays
    int64_t max_vox = 0;
    for (auto &s : active) {
        if (s->state != 1 || s->rounds_done >= s->rounds_total) continue;
        cyl_plan *pl = s->plan;
        const Part &pt = parts[s->req.part];
        const int subset = std::min(cfg.subset_size, s->req.n_proj);
        const int r = s->rounds_done;
        const int p0 = (r % s->n_sub) * subset;
        BatchScan sc{};
        sc.sd = pl->scan_dev();
        sc.rl = pl->ray_list();
        lists = lists || pl->use_list;
        sc.sino = s->d_sino;
        sc.x_proj = cfg.storage == CYL_F32 ? s->d_x : s->d_x32;   // the FP32 iterate
        sc.q[0] = pl->d_q;
        sc.q[1] = pl->d_q + (size_t)subset * pl->n_pix;
        sc.q_len = (int64_t)subset * pl->n_pix;
        sc.nd[0] = pl->d_nd[0];
        sc.nd[1] = pl->d_nd[1];
        sc.nd_len = pl->n_vox;
        sc.upd.x32 = cfg.storage == CYL_F32 ? static_cast<float *>(s->d_x) : s->d_x32;
        sc.upd.x16 = nullptr;               // the result is rounded once, at the end
        sc.upd.x16_t = cfg.storage;
        sc.upd.strict16 = 0;
        sc.upd.w = pt.d_w;
        sc.upd.w_t = (cyl_dtype)cfg.weight_dtype;
        sc.upd.wscale = pt.d_w ? pt.d_wscale : nullptr;
        sc.upd.lambda = (float)cfg.lambda;
        sc.upd.den_eps = sc.sd.g.eps;
        sc.upd.clamp = cfg.clamp_nonneg;
        items.push_back(BatchItem{(int)scans.size(), p0, std::min(subset, s->req.n_proj - p0), r & 1});
        scans.push_back(sc);
        members.push_back(s);
        max_vox = std::max(max_vox, pl->n_vox);
        if (!have_p) {
            fused = pl->fused;
            Pf = fused ? pl->p_sart : pl->p_fp;
            Pb = pl->p_bp;
            have_p = 1;
        }
    }
    if (scans.empty()) return CYL_OK;
    const int n = (int)scans.size();
    // descriptor slot: wait until the copy of its previous round has finished
    const int slot = next_slot;
    next_slot = (next_slot + 1) % n_slots;
    if (!wait_event(slot_ev[slot])) return set_error(CYL_ETIMEOUT, "round slot wait");
    char *h = static_cast<char *>(h_slot[slot]);
    char *d = static_cast<char *>(d_slot[slot]);
    const size_t b_scans = sizeof(BatchScan) * cfg.max_active, b_items = sizeof(BatchItem) * cfg.max_active;
    std::memcpy(h, scans.data(), sizeof(BatchScan) * n);
    std::memcpy(h + b_scans, items.data(), sizeof(BatchItem) * n);
    std::memcpy(h + b_scans + b_items, &n, sizeof(int));
    if (cudaMemcpyAsync(d, h, slot_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return set_error(CYL_EDEVICE, "round descriptors");
    if (cudaEventRecord(slot_ev[slot], st) != cudaSuccess) return set_error(CYL_EDEVICE, "event");
    cudaError_t e = launch_batch_round(reinterpret_cast<BatchScan *>(d), reinterpret_cast<BatchItem *>(d + b_scans),
                                       reinterpret_cast<int *>(d + b_scans + b_items), n, 0, max_vox, Pf, Pb,
                                       fused ? (kRoundFused | kRoundUpdate) : kRoundAll, d_sched, CYL_F32,
                                       cfg.storage, CYL_F32, st, lists);
    if (e != cudaSuccess) return cuda_error(e, "round launch");
    ++stats.rounds;
    for (auto &s : members) {
        if (++s->rounds_done == s->rounds_total) {
            if (cfg.storage != CYL_F32)
                launch_convert(s->d_x32, CYL_F32, s->d_x, cfg.storage, s->plan->n_vox, st);
            if (s->own_x)
                cudaMemcpyAsync(s->req.x_out, s->d_x, (size_t)s->plan->n_vox * dtype_size(cfg.storage),
                                cudaMemcpyDeviceToHost, st);
            cudaEventRecord(s->done_ev, st);
            s->state = 2;
        }
    }
    return CYL_OK;
}

void cyl_server::loop()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // admission, first come first served, by device footprint
        while (!queue.empty() && (int)active.size() < cfg.max_active) {
            auto s = queue.front();
            const Part &pt = parts[s->req.part];
            size_t plan_b = 0, scan_b = 0;
            footprint(pt, s->req.n_proj, s->angles.data(), s->req.pose, plan_b, scan_b);
            // an idle plan of the same part and views is reused: its bytes are counted
            const PlanKey key{s->req.part, s->req.n_proj, hash_angles(s->angles)};
            auto reuse = idle_plans.find(key);
            int64_t reuse_bytes = 0;
            if (reuse != idle_plans.end()) cyl_plan_sizes(reuse->second, nullptr, nullptr, nullptr, &reuse_bytes);
            const size_t fp = scan_b + std::max(plan_b, (size_t)reuse_bytes);
            if (hbm_in_use - reuse_bytes + (int64_t)fp > cfg.hbm_budget_bytes) {
                // evict another idle plan, or wait for running scans to finish
                auto it = idle_plans.begin();
                while (it != idle_plans.end() && it == reuse) ++it;
                if (it == idle_plans.end()) break;
                int64_t pb = 0;
                cyl_plan_sizes(it->second, nullptr, nullptr, nullptr, &pb);
                cyl_plan_destroy(it->second);
                idle_plans.erase(it);
                idle_bytes -= pb;
                hbm_in_use -= pb;
                continue;
            }
            if (reuse != idle_plans.end()) {     // admit() takes it from the pool
                idle_bytes -= reuse_bytes;
                hbm_in_use -= reuse_bytes;
            }
            queue.pop_front();
            s->bytes = fp;
            hbm_in_use += (int64_t)fp;
            s->t_admit = now_ns();
            s->state = 1;
            active.push_back(s);
            const int rc = admit(s);
            if (rc) {
                active.pop_back();
                finish(s, rc);
            }
        }
        if (active.empty()) {
            if (stop) break;
            cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        // rounds run with the lock released, so submissions and polls are not held up
        std::vector<std::shared_ptr<Scan>> snapshot = active;
        lk.unlock();
        int rc = CYL_OK;
        for (int k = 0; k < std::max(1, cfg.rounds_ahead) && rc == CYL_OK; ++k) rc = run_round();
        lk.lock();
        if (rc) {
            for (auto &s : snapshot)
                if (s->state == 1 || s->state == 2) finish(s, rc);
        }
        // retire scans whose result is out; block (bounded) only when nothing else runs
        bool runnable = false;
        for (auto &s : snapshot) runnable |= s->state == 1;
        for (auto &s : snapshot) {
            if (s->state != 2) continue;
            cudaError_t q = cudaEventQuery(s->done_ev);
            if (q == cudaErrorNotReady && !runnable && queue.empty()) {
                lk.unlock();
                const bool ok = wait_event(s->done_ev);
                lk.lock();
                q = ok ? cudaSuccess : cudaErrorLaunchTimeout;
            }
            if (q == cudaSuccess) finish(s, CYL_OK);
            else if (q != cudaErrorNotReady) finish(s, q == cudaErrorLaunchTimeout ? CYL_ETIMEOUT : CYL_EDEVICE);
        }
        active.erase(std::remove_if(active.begin(), active.end(),
                                    [](const std::shared_ptr<Scan> &s) { return s->state == 3; }),
                     active.end());
    }
    // shutdown: queued requests are cancelled
    for (auto &s : queue) {
        s->status = CYL_ECANCELLED;
        s->state = 3;
    }
    queue.clear();
    done_cv.notify_all();
}

// ------------------------------------------------------------------------------ ABI

extern "C" int cyl_server_create(const cyl_server_cfg *cfg, cyl_server **out)
{
    if (!cfg || !out) return set_error(CYL_EINVAL, "cfg or out is null");
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->max_active < 1 || cfg->max_active > 1024 ||
        cfg->n_iter < 0 || cfg->subset_size < 1 || !std::isfinite(cfg->lambda) ||
        (cfg->weight_mode != 0 && cfg->weight_mode != 1) || cfg->storage < CYL_F32 ||
        cfg->storage > CYL_BF16 || cfg->rounds_ahead < 0 || cfg->rounds_ahead > 64 ||
        !valid_weight_dtype(cfg->weight_dtype))
        return set_error(CYL_EINVAL, "bad server configuration");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return set_error(CYL_EDEVICE, "no such CUDA device");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(cfg->device);
    cyl_server *s = new (std::nothrow) cyl_server();
    if (!s) return set_error(CYL_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    if (s->cfg.rounds_ahead == 0) s->cfg.rounds_ahead = 4;
    int rc = CYL_OK;
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) rc = set_error(CYL_EDEVICE, "stream");
    s->n_slots = s->cfg.rounds_ahead + 2;
    s->slot_bytes = (sizeof(BatchScan) + sizeof(BatchItem)) * s->cfg.max_active + 16;
    for (int k = 0; k < s->n_slots && !rc; ++k) {
        void *h = nullptr, *d = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaMallocHost(&h, s->slot_bytes) != cudaSuccess || cudaMalloc(&d, s->slot_bytes) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            rc = set_error(CYL_ENOMEM, "round descriptor slots");
        s->h_slot.push_back(h);
        s->d_slot.push_back(d);
        s->slot_ev.push_back(e);
    }
    if (!rc && (cudaMalloc(&s->d_sched, sizeof(int) * kSched) != cudaSuccess ||
                cudaMemset(s->d_sched, 0, sizeof(int) * kSched) != cudaSuccess))
        rc = set_error(CYL_ENOMEM, "scheduler state");
    if (rc) {
        cyl_server_destroy(s);
        if (prev >= 0) cudaSetDevice(prev);
        return rc;
    }
    s->thr = std::thread([s] { s->loop(); });
    if (prev >= 0) cudaSetDevice(prev);
    *out = s;
    return CYL_OK;
}

extern "C" int cyl_server_add_part(cyl_server *srv, const cyl_grid *grid, const cyl_geom *geom,
                                   const void *x0, const void *w, int32_t *part)
{
    if (!srv || !grid || !geom || !part) return set_error(CYL_EINVAL, "null argument");
    if (geom->frames_mm) return set_error(CYL_EINVAL, "the server takes circular scans only");
    // validate with a one-view stand-in for the per-request angles
    const double zero = 0.0;
    cyl_geom g1 = *geom;
    g1.n_proj = 1;
    g1.angles_rad = &zero;
    const cyl_pose p0{0, 0, 0, 0, 0, 0};
    int rc = validate_scan(grid, &g1, &p0);
    if (rc) return rc;
    {   // a round of max_active scans counts its warp tasks in 32 bits (16 pieces per ray)
        const int64_t sub = srv->cfg.subset_size;
        const int64_t per = ((sub * geom->det_w * geom->det_h + 31) / 32) * kSplit + kSplit;
        if (per * srv->cfg.max_active >= ((int64_t)1 << 31) - 1)
            return set_error(CYL_EINVAL, "part too large for rounds of max_active scans (2^31 warp tasks)");
    }
    Part pt;
    pt.grid = *grid;
    pt.geom = g1;
    pt.geom.angles_rad = nullptr;
    pt.n_vox = (int64_t)grid->n_h * grid->n_theta * grid->n_r;
    const size_t sb = dtype_size(srv->cfg.storage);
    const cyl_dtype w_t = (cyl_dtype)srv->cfg.weight_dtype;
    const size_t wb = dtype_size(w_t);
    pt.bytes = (size_t)pt.n_vox * sb + (w ? (size_t)pt.n_vox * wb : 0) + 2 * sizeof(float);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->cfg.device);
    struct Restore {
        int d;
        ~Restore() { if (d >= 0) cudaSetDevice(d); }
    } restore{prev};
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->hbm_in_use + (int64_t)pt.bytes > srv->cfg.hbm_budget_bytes)
        return set_error(CYL_EADMIT, "part data exceeds the HBM budget");
    if (x0 && cudaMalloc(&pt.d_x0, (size_t)pt.n_vox * sb) != cudaSuccess) return set_error(CYL_ENOMEM, "warm start");
    if (w && cudaMalloc(&pt.d_w, (size_t)pt.n_vox * wb) != cudaSuccess) return set_error(CYL_ENOMEM, "weights");
    if (cudaMalloc(&pt.d_wscale, 2 * sizeof(float)) != cudaSuccess) return set_error(CYL_ENOMEM, "weight scale");
    if (x0 && cudaMemcpyAsync(pt.d_x0, x0, (size_t)pt.n_vox * sb, cudaMemcpyDefault, srv->st) != cudaSuccess)
        return set_error(CYL_EDEVICE, "warm start copy");
    if (w) {
        if (cudaMemcpyAsync(pt.d_w, w, (size_t)pt.n_vox * wb, cudaMemcpyDefault, srv->st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "weight copy");
        if (launch_weight_scale(pt.d_w, w_t, pt.n_vox, srv->cfg.weight_mode, (float)srv->cfg.lambda, pt.d_wscale,
                                srv->st) != cudaSuccess)
            return set_error(CYL_EDEVICE, "weight scale");
    }
    if (cudaStreamSynchronize(srv->st) != cudaSuccess) return set_error(CYL_EDEVICE, "part upload");
    srv->hbm_in_use += (int64_t)pt.bytes;
    srv->parts.push_back(pt);
    *part = (int32_t)srv->parts.size() - 1;
    return CYL_OK;
}

extern "C" int cyl_submit(cyl_server *srv, const cyl_request *req, uint64_t *ticket)
{
    if (!srv || !req || !ticket) return set_error(CYL_EINVAL, "null argument");
    auto s = std::make_shared<Scan>();
    s->req = *req;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return set_error(CYL_ECANCELLED, "server is shutting down");
        if (req->part < 0 || req->part >= (int)srv->parts.size()) return set_error(CYL_EINVAL, "unknown part");
        if (req->n_proj < 1 || !req->angles_rad || !req->sino || !req->x_out)
            return set_error(CYL_EINVAL, "request needs views, angles, sinogram and output");
        const Part &pt = srv->parts[req->part];
        cyl_geom g = pt.geom;
        g.n_proj = req->n_proj;
        g.angles_rad = req->angles_rad;
        int rc = validate_scan(&pt.grid, &g, &req->pose);
        if (rc) return rc;
        int64_t part_bytes = 0;
        for (const Part &p : srv->parts) part_bytes += (int64_t)p.bytes;
        size_t plan_b = 0, scan_b = 0;
        srv->footprint(pt, req->n_proj, req->angles_rad, req->pose, plan_b, scan_b);
        if (part_bytes + (int64_t)(plan_b + scan_b) > srv->cfg.hbm_budget_bytes)
            return set_error(CYL_EADMIT, "the scan can never fit the HBM budget");
        s->angles.assign(req->angles_rad, req->angles_rad + req->n_proj);
        s->req.angles_rad = s->angles.data();
        s->ticket = srv->next_ticket++;
        s->t_submit = now_ns();
        srv->queue.push_back(s);
        srv->tickets[s->ticket] = s;
        ++srv->stats.submitted;
        *ticket = s->ticket;
    }
    srv->cv.notify_one();
    return CYL_OK;
}

static int fill_result(cyl_server *srv, std::map<uint64_t, std::shared_ptr<Scan>>::iterator it, cyl_result *out)
{
    Scan &s = *it->second;
    if (out) {
        out->status = s.state == 3 ? s.status : CYL_EPENDING;
        out->submit_ns = s.t_submit;
        out->admit_ns = s.t_admit;
        out->done_ns = s.t_done;
    }
    if (s.state != 3) return CYL_EPENDING;
    const int st = s.status;
    srv->tickets.erase(it);
    return st;
}

extern "C" int cyl_poll(cyl_server *srv, uint64_t ticket, cyl_result *out)
{
    if (!srv) return set_error(CYL_EINVAL, "server is null");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return set_error(CYL_ENOTFOUND, "unknown ticket");
    return fill_result(srv, it, out);
}

extern "C" int cyl_wait(cyl_server *srv, uint64_t ticket, int64_t timeout_ms, cyl_result *out)
{
    if (!srv || timeout_ms < 0) return set_error(CYL_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->tickets.find(ticket);
        if (it == srv->tickets.end()) return set_error(CYL_ENOTFOUND, "unknown ticket");
        if (it->second->state == 3) return fill_result(srv, it, out);
        if (srv->done_cv.wait_until(lk, until) == std::cv_status::timeout) {
            it = srv->tickets.find(ticket);
            if (it != srv->tickets.end() && it->second->state == 3) return fill_result(srv, it, out);
            if (out && it != srv->tickets.end()) fill_result(srv, it, out);
            return set_error(CYL_ETIMEOUT, "still pending");
        }
    }
}

extern "C" int cyl_server_get_stats(cyl_server *srv, cyl_server_stats *out)
{
    if (!srv || !out) return set_error(CYL_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->active = (int64_t)srv->active.size();
    out->queued = (int64_t)srv->queue.size();
    out->hbm_in_use = srv->hbm_in_use;
    return CYL_OK;
}

extern "C" int cyl_server_destroy(cyl_server *srv)
{
    if (!srv) return CYL_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (auto &s : srv->queue) {
            s->status = CYL_ECANCELLED;
            s->state = 3;
        }
        srv->queue.clear();
    }
    srv->cv.notify_all();
    if (srv->thr.joinable()) srv->thr.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->cfg.device);
    if (srv->st) cudaStreamSynchronize(srv->st);
    for (auto &kv : srv->idle_plans) cyl_plan_destroy(kv.second);
    for (Part &p : srv->parts) {
        cudaFree(p.d_x0);
        cudaFree(p.d_w);
        cudaFree(p.d_wscale);
    }
    for (size_t k = 0; k < srv->h_slot.size(); ++k) {
        if (srv->h_slot[k]) cudaFreeHost(srv->h_slot[k]);
        if (srv->d_slot[k]) cudaFree(srv->d_slot[k]);
        if (srv->slot_ev[k]) cudaEventDestroy(srv->slot_ev[k]);
    }
    if (srv->d_sched) cudaFree(srv->d_sched);
    if (srv->st) cudaStreamDestroy(srv->st);
    if (prev >= 0) cudaSetDevice(prev);
    delete srv;
    return CYL_OK;
}
